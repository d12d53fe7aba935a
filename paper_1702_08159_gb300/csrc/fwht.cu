// Standalone batched in-place unnormalised Walsh-Hadamard transform
// (Sec. "Fast Walsh Hadamard"; the paper's Sec. "Implementation of Fast Walsh
// Hadamard" splits a large transform into passes over memory down to an
// in-cache routine -- here the "cache" is registers plus shared memory).
//
// Regimes, by L = log2 d:
//   L = 1..4    one thread per vector, entirely in registers.
//   L = 5..10   a group of 2^(L-5) lanes per vector (32/2^(L-5) vectors per
//               warp): register phases A and B with one shared-memory layout
//               move in between, 128-bit coalesced global loads and stores.
//   L = 11..15  one block of 2^(L-10) warps per vector: each warp transforms
//               a 1024-float chunk like the d = 1024 kernel, then one
//               shared-memory exchange carries index bits 10..L-1.
//   L = 16, 17  one pass: a thread-block cluster of 2^(L-15) blocks per
//               vector; each block transforms a 2^15 slice that way, then
//               the rank bits are transformed across the cluster through
//               distributed shared memory on the way out to HBM.
//   L = 18..20  two passes over HBM: the L = 15 kernel on every 2^15 block
//               (index bits 0..14), then a column pass over bits 15..L-1.
// Every element is read and written once per pass.
#include <cooperative_groups.h>
#include <cuda_runtime.h>

#include <algorithm>

#include "common.cuh"
#include "internal.h"

namespace mck {
namespace {

namespace cg = cooperative_groups;

constexpr int kWarpsPerBlock = 4;

template <int L>
__global__ void __launch_bounds__(128) k_fwht_tiny(float* __restrict__ x, int64_t n) {
  constexpr int d = 1 << L;
  for (int64_t v = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; v < n;
       v += (int64_t)gridDim.x * blockDim.x) {
    float w[d];
    float* p = x + v * d;
#pragma unroll
    for (int k = 0; k < d; ++k) w[k] = p[k];
#pragma unroll
    for (int h = 1; h < d; h <<= 1)
#pragma unroll
      for (int k = 0; k < d; ++k)
        if (!(k & h)) {
          const float a = w[k], c = w[k | h];
          w[k] = a + c;
          w[k | h] = a - c;
        }
#pragma unroll
    for (int k = 0; k < d; ++k) p[k] = w[k];
  }
}

template <int L>
__device__ __forceinline__ void gload_A(const float* __restrict__ row, int lam, bool valid,
                                        float (&w)[32]) {
#pragma unroll
  for (int m = 0; m < 8; ++m) {
    float4 v = make_float4(0.f, 0.f, 0.f, 0.f);
    if (valid) v = __ldcs(reinterpret_cast<const float4*>(row + Lay<L>::kA(lam, 4 * m)));
    w[4 * m] = v.x;
    w[4 * m + 1] = v.y;
    w[4 * m + 2] = v.z;
    w[4 * m + 3] = v.w;
  }
}

template <int L>
__device__ __forceinline__ void gstore_A(float* __restrict__ row, int lam, const float (&w)[32]) {
#pragma unroll
  for (int m = 0; m < 8; ++m)
    __stcs(reinterpret_cast<float4*>(row + Lay<L>::kA(lam, 4 * m)),
           make_float4(w[4 * m], w[4 * m + 1], w[4 * m + 2], w[4 * m + 3]));
}

template <int L>
__global__ void __launch_bounds__(kWarpsPerBlock * 32) k_fwht_warp(float* __restrict__ x,
                                                                    int64_t n) {
  using Y = Lay<L>;
  constexpr int VPW = 32 / Y::T;
  __shared__ __align__(16) float sm[kWarpsPerBlock][VPW * Y::SLOT];
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int g = lane / Y::T, lam = lane % Y::T;
  float* buf = sm[warp];
  const int64_t groups = (n + VPW - 1) / VPW;
  for (int64_t grp = (int64_t)blockIdx.x * kWarpsPerBlock + warp; grp < groups;
       grp += (int64_t)gridDim.x * kWarpsPerBlock) {
    const int64_t v = grp * VPW + g;
    const bool valid = v < n;
    float* row = x + v * Y::d;
    float w[32];
    gload_A<L>(row, lam, valid, w);
    hreg<Y::maskA()>(w);
    if constexpr (L > 5) {
      store_A<L>(buf, g, lam, w);
      __syncwarp();
      load_B<L>(buf, g, lam, w);
    }
    hreg<Y::maskB()>(w);
    if constexpr (L > 5) {
      // A thread rewrites exactly the slots it just read, so no barrier is
      // needed between a load phase and the next store phase.
      store_B<L>(buf, g, lam, w);
      __syncwarp();
      load_A<L>(buf, g, lam, w);
    }
    if (valid) gstore_A<L>(row, lam, w);
  }
}

// One block of W = 2^(L-10) warps per vector (11 <= L <= 15). Warp w
// transforms chunk w (index bits 0..9) exactly like the d = 1024 warp kernel,
// leaving it in natural order in its own 1056-word slot of shared memory;
// after one block barrier thread j takes columns c = j, j + 32W, ...
// (32/W of them) with their W values at stride 1024 and applies H_W over
// index bits 10..L-1 in registers on the way out to HBM (coalesced).
template <int L>
__global__ void __launch_bounds__(1 << (L - 5)) k_fwht_chunks(float* __restrict__ x, int64_t n) {
  using Y = Lay<10>;
  constexpr int W = 1 << (L - 10), NT = 32 * W, CPT = 32 / W;
  extern __shared__ float4 sm4[];
  float* sm = reinterpret_cast<float*>(sm4);
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  float* buf = sm + warp * Y::SLOT;
  for (int64_t v = blockIdx.x; v < n; v += gridDim.x) {
    float* row = x + (v << L);
    {
      float w[32];
      gload_A<10>(row + warp * 1024, lane, true, w);
      hreg<Y::maskA()>(w);
      store_A<10>(buf, 0, lane, w);
      __syncwarp();
      load_B<10>(buf, 0, lane, w);
      hreg<Y::maskB()>(w);
      __syncwarp();
      store_B<10>(buf, 0, lane, w);
    }
    __syncthreads();
    // At 2^15 (one block per SM) this block's next vector goes into L2 while
    // the current one is transformed: 0.381 -> 0.355 ms per GiB; at 2^11..2^14
    // several blocks share an SM and the prefetch only competed for HBM
    // (0.351 -> 0.373 ms), so it is left out there.
    if constexpr (L == 15)
      if (v + gridDim.x < n && lane == 0)
        prefetch_l2_bulk(row + ((int64_t)gridDim.x << L) + warp * 1024, 4096u);
#pragma unroll
    for (int j = 0; j < CPT; ++j) {
      const int c = threadIdx.x + NT * j;
      float u[W];
#pragma unroll
      for (int i = 0; i < W; ++i) u[i] = sm[i * Y::SLOT + pad(c)];
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
    __syncthreads();  // the slots are read before the next vector overwrites them
  }
}

// Column pass of the two-pass regime: H over index bits 15..L-1 of each
// vector. Thread t of vector v handles column c = t (mod 2^15): the R = 2^(L-15)
// elements c + 2^15 i, i < R, kept in registers. Consecutive threads read
// consecutive columns (coalesced).
template <int R>
__global__ void __launch_bounds__(256) k_fwht_columns(float* __restrict__ x, int64_t n) {
  constexpr int64_t kBlock = 1 << 15;
  const int64_t total = n * kBlock;
  for (int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; t < total;
       t += (int64_t)gridDim.x * blockDim.x) {
    const int64_t v = t / kBlock, c = t % kBlock;
    float* p = x + v * kBlock * R + c;
    float w[R];
#pragma unroll
    for (int i = 0; i < R; ++i) w[i] = __ldcs(p + i * kBlock);
#pragma unroll
    for (int h = 1; h < R; h <<= 1)
#pragma unroll
      for (int i = 0; i < R; ++i)
        if (!(i & h)) {
          const float a = w[i], b = w[i | h];
          w[i] = a + b;
          w[i | h] = a - b;
        }
#pragma unroll
    for (int i = 0; i < R; ++i) __stcs(p + i * kBlock, w[i]);
  }
}

// One vector of 2^(LS + log2 CS) per thread-block cluster of CS blocks
// (single pass over HBM). Block r of the cluster loads slice r (index bits
// 0..LS-1 local, bits LS.. = r) and transforms the local bits as the chunked
// block kernel does (bits 0..9 per warp, then 10..LS-1 across the chunks),
// leaving the slice in shared memory. After a cluster barrier, block r takes
// 1/CS of the local indices, four consecutive at a time: it reads the CS
// slices' values there through distributed shared memory (128-bit), applies
// H_CS (the rank bits) and writes the CS results to HBM (128-bit,
// coalesced). A second cluster barrier keeps the slices alive until every
// block has read them.
template <int LS, int CS>
__global__ void __launch_bounds__(1 << (LS - 5)) k_fwht_cluster(float* __restrict__ x, int64_t n) {
  using Y = Lay<10>;
  constexpr int S = 1 << LS, W = 1 << (LS - 10), NT = 32 * W, CPT = 32 / W;
  constexpr int OWN = S / CS, PER4 = OWN / (4 * NT);
  static_assert(LS >= 11 && LS <= 15 && PER4 >= 1 && PER4 * 4 * NT * CS == S,
                "cluster slices (2 <= CS <= 8)");
  extern __shared__ float4 sm4[];
  float* sm = reinterpret_cast<float*>(sm4);  // W slots of 1056 words: chunk i at i * SLOT + pad(c)
  cg::cluster_group cl = cg::this_cluster();
  const int r = (int)cl.block_rank();
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  float* buf = sm + warp * Y::SLOT;
  const int64_t ncl = gridDim.x / CS;
  for (int64_t v = blockIdx.x / CS; v < n; v += ncl) {
    float* row = x + v * (int64_t)(S * CS);
    // index bits 0..9: warp w transforms chunk w of the slice in registers
    {
      float w[32];
      gload_A<10>(row + (int64_t)r * S + warp * 1024, lane, true, w);
      hreg<Y::maskA()>(w);
      store_A<10>(buf, 0, lane, w);
      __syncwarp();
      load_B<10>(buf, 0, lane, w);
      hreg<Y::maskB()>(w);
      __syncwarp();
      store_B<10>(buf, 0, lane, w);
    }
    __syncthreads();
    // The cluster's next vector: this warp's chunk of it into L2 while the
    // current one is transformed and exchanged (issued after this vector's
    // loads, so as not to compete with them): 2^16 0.531 -> 0.490 ms, 2^17
    // 0.614 -> 0.579 ms.
    if (v + ncl < n && lane == 0)
      prefetch_l2_bulk(row + ncl * (int64_t)(S * CS) + (int64_t)r * S + warp * 1024, 4096u);
    // index bits 10..LS-1: across the slice's chunks, in place
#pragma unroll
    for (int j = 0; j < CPT; ++j) {
      const int c = threadIdx.x + NT * j;
      float u[W];
#pragma unroll
      for (int i = 0; i < W; ++i) u[i] = sm[i * Y::SLOT + pad(c)];
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
      for (int i = 0; i < W; ++i) sm[i * Y::SLOT + pad(c)] = u[i];
    }
    cl.sync();  // every slice is transformed over its local bits
    // rank bits: block r takes local indices [r OWN, (r+1) OWN), four at a time
#pragma unroll
    for (int q = 0; q < PER4; ++q) {
      const int i = r * OWN + 4 * (q * NT + (int)threadIdx.x);
      const int at = (i >> 10) * Y::SLOT + pad(i & 1023);  // 4 consecutive words
      float4 u[CS];
#pragma unroll
      for (int c = 0; c < CS; ++c)
        u[c] = *reinterpret_cast<const float4*>(cl.map_shared_rank(sm, c) + at);
#pragma unroll
      for (int h = 1; h < CS; h <<= 1)
#pragma unroll
        for (int c = 0; c < CS; ++c)
          if (!(c & h)) {
            const float4 a = u[c], b = u[c | h];
            u[c] = make_float4(a.x + b.x, a.y + b.y, a.z + b.z, a.w + b.w);
            u[c | h] = make_float4(a.x - b.x, a.y - b.y, a.z - b.z, a.w - b.w);
          }
#pragma unroll
      for (int c = 0; c < CS; ++c)
        __stcs(reinterpret_cast<float4*>(row + (int64_t)c * S + i), u[c]);
    }
    cl.sync();  // no slice is overwritten while another block still reads it
  }
}

template <class K>
int occupancy_blocks(K kernel, int threads, size_t smem) {
  int b = 0;
  if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&b, kernel, threads, smem) != cudaSuccess)
    b = 1;
  return std::max(b, 1);
}

inline unsigned grid_for(int64_t work, int per_block, int num_sms, int occ) {
  const int64_t need = (work + per_block - 1) / per_block;
  const int64_t cap = (int64_t)num_sms * occ;
  return (unsigned)std::max<int64_t>(1, std::min(need, cap));
}

template <int L>
cudaError_t run_tiny(float* x, int64_t n, int num_sms, cudaStream_t s) {
  const int occ = occupancy_blocks(k_fwht_tiny<L>, 128, 0);
  k_fwht_tiny<L><<<grid_for(n, 128, num_sms, occ), 128, 0, s>>>(x, n);
  return cudaGetLastError();
}

template <int L>
cudaError_t run_warp(float* x, int64_t n, int num_sms, cudaStream_t s) {
  constexpr int VPW = 32 / Lay<L>::T;
  const int occ = occupancy_blocks(k_fwht_warp<L>, kWarpsPerBlock * 32, 0);
  k_fwht_warp<L><<<grid_for(n, VPW * kWarpsPerBlock, num_sms, occ), kWarpsPerBlock * 32, 0,
                   s>>>(x, n);
  return cudaGetLastError();
}

template <int L>
cudaError_t run_chunks(float* x, int64_t n, int num_sms, cudaStream_t s) {
  const size_t smem = sizeof(float) * ((size_t)Lay<10>::SLOT << (L - 10));
  cudaError_t err =
      cudaFuncSetAttribute(k_fwht_chunks<L>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (err != cudaSuccess) return err;
  const int occ = occupancy_blocks(k_fwht_chunks<L>, 1 << (L - 5), smem);
  k_fwht_chunks<L><<<grid_for(n, 1, num_sms, occ), 1 << (L - 5), smem, s>>>(x, n);
  return cudaGetLastError();
}

template <int R>
cudaError_t run_columns(float* x, int64_t n, int num_sms, cudaStream_t s) {
  const int occ = occupancy_blocks(k_fwht_columns<R>, 256, 0);
  k_fwht_columns<R><<<grid_for(n << 15, 256, num_sms, occ), 256, 0, s>>>(x, n);
  return cudaGetLastError();
}

template <int LS, int CS>
cudaError_t run_cluster(float* x, int64_t n, cudaStream_t s) {
  auto kern = k_fwht_cluster<LS, CS>;
  const size_t smem = sizeof(float) * ((size_t)Lay<10>::SLOT << (LS - 10));
  cudaError_t err = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (err != cudaSuccess) return err;
  if (CS > 8) {
    err = cudaFuncSetAttribute(kern, cudaFuncAttributeNonPortableClusterSizeAllowed, 1);
    if (err != cudaSuccess) return err;
  }
  cudaLaunchConfig_t cfg{};
  cfg.blockDim = dim3(Lay<LS>::T, 1, 1);
  cfg.dynamicSmemBytes = smem;
  cfg.stream = s;
  cudaLaunchAttribute attr[1];
  attr[0].id = cudaLaunchAttributeClusterDimension;
  attr[0].val.clusterDim.x = CS;
  attr[0].val.clusterDim.y = 1;
  attr[0].val.clusterDim.z = 1;
  cfg.attrs = attr;
  cfg.numAttrs = 1;
  cfg.gridDim = dim3(CS, 1, 1);
  int clusters = 0;
  if (cudaOccupancyMaxActiveClusters(&clusters, kern, &cfg) != cudaSuccess || clusters < 1) {
    cudaGetLastError();
    return cudaErrorInvalidConfiguration;
  }
  cfg.gridDim = dim3((unsigned)(CS * std::min<int64_t>(n, clusters)), 1, 1);
  err = cudaLaunchKernelEx(&cfg, kern, x, n);
  if (err != cudaSuccess) return err;
  return cudaGetLastError();
}

}  // namespace

cudaError_t launch_fwht_high_bits(float* x, int64_t n, int L, int num_sms, cudaStream_t s) {
  if (n == 0 || L <= 15) return cudaSuccess;
  // bits 15..L-1 at stride 2^15
  switch (L) {
    case 16: return run_columns<2>(x, n, num_sms, s);
    case 17: return run_columns<4>(x, n, num_sms, s);
    case 18: return run_columns<8>(x, n, num_sms, s);
    case 19: return run_columns<16>(x, n, num_sms, s);
    default: return run_columns<32>(x, n, num_sms, s);
  }
}

cudaError_t launch_fwht(float* x, int64_t n, int L, int num_sms, cudaStream_t s, int regime) {
  if (n == 0 || L == 0) return cudaSuccess;
  switch (L) {
    case 1: return run_tiny<1>(x, n, num_sms, s);
    case 2: return run_tiny<2>(x, n, num_sms, s);
    case 3: return run_tiny<3>(x, n, num_sms, s);
    case 4: return run_tiny<4>(x, n, num_sms, s);
    case 5: return run_warp<5>(x, n, num_sms, s);
    case 6: return run_warp<6>(x, n, num_sms, s);
    case 7: return run_warp<7>(x, n, num_sms, s);
    case 8: return run_warp<8>(x, n, num_sms, s);
    case 9: return run_warp<9>(x, n, num_sms, s);
    case 10: return run_warp<10>(x, n, num_sms, s);
    case 11: return run_chunks<11>(x, n, num_sms, s);
    case 12: return run_chunks<12>(x, n, num_sms, s);
    case 13: return run_chunks<13>(x, n, num_sms, s);
    case 14: return run_chunks<14>(x, n, num_sms, s);
    case 15: return run_chunks<15>(x, n, num_sms, s);
    default: break;
  }
  if (L > 20) return cudaErrorInvalidValue;
  // One pass on a cluster of 2 or 4 blocks of 2^15 (54% and 49% of the copy
  // bandwidth, against 33% and 37% for two passes) unless the caller picks
  // another regime (MCK_FWHT_CLUSTER_2_14: clusters of 4 or 8 blocks of 2^14,
  // MCK_FWHT_TWO_PASS); a cluster of 8 whole-SM blocks packs the GPCs poorly
  // and measured slower than two passes.
  if (L <= 17 && regime != MCK_FWHT_TWO_PASS) {
    if (regime == MCK_FWHT_CLUSTER_2_14)
      return L == 16 ? run_cluster<14, 4>(x, n, s) : run_cluster<14, 8>(x, n, s);
    return L == 16 ? run_cluster<15, 2>(x, n, s) : run_cluster<15, 4>(x, n, s);
  }
  const int64_t blocks = n << (L - 15);
  cudaError_t err = run_chunks<15>(x, blocks, num_sms, s);
  if (err != cudaSuccess) return err;
  switch (L) {
    case 16: return run_columns<2>(x, n, num_sms, s);
    case 17: return run_columns<4>(x, n, num_sms, s);
    case 18: return run_columns<8>(x, n, num_sms, s);
    case 19: return run_columns<16>(x, n, num_sms, s);
    default: return run_columns<32>(x, n, num_sms, s);
  }
}

}  // namespace mck
