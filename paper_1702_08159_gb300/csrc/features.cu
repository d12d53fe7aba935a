// Fused Fastfood feature kernels: for each sample n and expansion e,
//
//   u  = H (B_e x-hat)        x-hat = x padded with zeros to d   (Eq. etn:mckernel)
//   v  = Pi_e u               v_k = u_{pi_e(k)}
//   h  = H (G_e v)
//   z  = Cs_e h               Cs = C/(sigma sqrt d)
//   phi[n, e] = [cos z | sin z]                                  (Eq. etn:mcfeatures)
//
// in one pass: x is read, the two transforms, the permutation and the
// diagonals run in registers and shared memory, and only phi is written
// (MODE_FEATURES) -- or phi is contracted with the classifier weights on the
// fly and only per-(sample, expansion) partial logits are written
// (MODE_LOGITS; Sec. "Empirical Analysis": softmax(W phi + b)).
//
// Kernels by L = log2 d:
//   L = 5..10  warp kernel. 2^(L-5) lanes hold one vector (32 registers
//              each); a warp processes 32/2^(L-5) samples at once. Work items
//              are (tile of samples, expansion); a warp loads the expansion's
//              tables into registers once per item (B as a bit mask, G, Cs and
//              the gather offsets of Pi, packed two per register) and runs
//              the item's samples.
//   L = 11..14 chunked block kernel (features): 2^(L-10) warps per (sample,
//              e), each transforming a 1024-float chunk like the warp kernel,
//              index bits 10..L-1 and the Pi gather through shared memory.
//   L = 11..15 block kernel: one block of 2^(L-5) threads per (sample, e)
//              (fused logits at these d, and features at d = 2^15).
//   L = 1..4   one thread per (sample, e).
#include <cuda_runtime.h>

#include <algorithm>

#include "common.cuh"
#include "internal.h"
#include "mma_h16.cuh"

namespace mck {
namespace {

constexpr int MODE_FEATURES = 0;
constexpr int MODE_LOGITS = 1;
// One warp per block: with 128 registers a thread, 16 single-warp blocks fit
// on an SM, the most residency the register file allows while the tables of
// one expansion stay in registers.
constexpr int kWarps = 1;
constexpr int kWarpMinBlocks = 14;  // feature mode; the logits mode keeps its accumulators unspilled
constexpr int CMAX = MCK_MAX_CLASSES;

struct Launch {
  FeatureArgs a;
  bool vec_x;         // x rows 16-byte aligned and in_dim % 4 == 0
  float* phi;         // MODE_FEATURES: n x 2Ed
  const float* W;     // MODE_LOGITS: C x 2Ed
  float* part;        // MODE_LOGITS: n x E x C
  int C;
  const uint4* wf;    // tensor-core logits: fp16 hi/lo fragments of the scaled W
  const float* winv;  // tensor-core logits: the per-class inverse scales
};

// Flip the sign of register j where bit j of `mask` is set (B = -1).
__device__ __forceinline__ void apply_signs(float (&w)[32], uint32_t mask) {
#pragma unroll
  for (int j = 0; j < 32; ++j)
    w[j] = __int_as_float(__float_as_int(w[j]) ^ ((mask << (31 - j)) & 0x80000000u));
}

// d = 1024: u into the skewed slot for the Pi gather (register j at word
// base + 33 j; see mck_plan_s::permS), and the lane's 16 packed gather
// offsets (byte offsets of registers 2i and 2i + 1 in the halves of word i).
__device__ __forceinline__ void store_skew(float* buf, uint32_t base, const float (&w)[32]) {
  float* q = buf + base;
#pragma unroll
  for (int j = 0; j < 32; ++j) q[33 * j] = w[j];
}
__device__ __forceinline__ void load_skew_offsets(const uint32_t* __restrict__ permS, int lam,
                                                  uint32_t (&poff)[16]) {
  const uint4* ps = reinterpret_cast<const uint4*>(permS) + lam;
#pragma unroll
  for (int q = 0; q < 4; ++q) {
    const uint4 v = __ldg(ps + q * 32);
    poff[4 * q] = v.x;
    poff[4 * q + 1] = v.y;
    poff[4 * q + 2] = v.z;
    poff[4 * q + 3] = v.w;
  }
}

// B bits of the elements of layout A held by thread lam, as a 32-bit mask.
template <int L>
__device__ __forceinline__ uint32_t load_bmask_A(const uint32_t* __restrict__ Bw, int lam) {
  uint32_t mask = 0;
#pragma unroll
  for (int m = 0; m < 8; ++m) {
    const int k0 = Lay<L>::kA(lam, 4 * m);  // multiple of 4: the 4 bits share a word
    mask |= ((__ldg(Bw + (k0 >> 5)) >> (k0 & 31)) & 0xFu) << (4 * m);
  }
  return mask;
}

// x-hat in layout A (zero past in_dim, zero for an invalid sample).
template <int L>
__device__ __forceinline__ void load_x_A(const Launch& P, int64_t n, bool valid, int lam,
                                         float (&w)[32]) {
  const float* row = P.a.x + n * P.a.ldx;
  const int64_t in_dim = P.a.in_dim;
#pragma unroll
  for (int m = 0; m < 8; ++m) {
    const int k0 = Lay<L>::kA(lam, 4 * m);
    float4 v = make_float4(0.f, 0.f, 0.f, 0.f);
    if (valid) {
      if (P.vec_x) {
        if (k0 < in_dim) v = __ldg(reinterpret_cast<const float4*>(row + k0));
      } else {
        if (k0 + 0 < in_dim) v.x = __ldg(row + k0 + 0);
        if (k0 + 1 < in_dim) v.y = __ldg(row + k0 + 1);
        if (k0 + 2 < in_dim) v.z = __ldg(row + k0 + 2);
        if (k0 + 3 < in_dim) v.w = __ldg(row + k0 + 3);
      }
    }
    w[4 * m] = v.x;
    w[4 * m + 1] = v.y;
    w[4 * m + 2] = v.z;
    w[4 * m + 3] = v.w;
  }
}

// Epilogue on layout A: z = Cs h, then either store [cos | sin] or fold them
// into the per-class partial sums acc[c] += <W_c, phi>.
template <int L, int MODE>
__device__ __forceinline__ void epilogue_A(const Launch& P, int64_t n, int e, bool valid, int lam,
                                           const float (&h)[32], const float (&cs)[32],
                                           float (&acc)[CMAX]) {
  constexpr int d = 1 << L;
  const int64_t F = 2ll * P.a.E * d;
#pragma unroll
  for (int m = 0; m < 8; ++m) {
    const int k0 = Lay<L>::kA(lam, 4 * m);
    float c[4], s[4];
    cos_sin4(&cs[4 * m], &h[4 * m], c, s);
    if constexpr (MODE == MODE_FEATURES) {
      if (valid) {
        float* o = P.phi + n * F + 2ll * e * d + k0;
        __stcs(reinterpret_cast<float4*>(o), make_float4(c[0], c[1], c[2], c[3]));
        __stcs(reinterpret_cast<float4*>(o + d), make_float4(s[0], s[1], s[2], s[3]));
      }
    } else {
      const float* wr = P.W + 2ll * e * d + k0;
#pragma unroll
      for (int cl = 0; cl < CMAX; ++cl) {
        if (cl < P.C) {
          const float4 wc = __ldg(reinterpret_cast<const float4*>(wr + cl * F));
          const float4 ws = __ldg(reinterpret_cast<const float4*>(wr + cl * F + d));
          float t = acc[cl];
          t = fmaf(wc.x, c[0], t);
          t = fmaf(wc.y, c[1], t);
          t = fmaf(wc.z, c[2], t);
          t = fmaf(wc.w, c[3], t);
          t = fmaf(ws.x, s[0], t);
          t = fmaf(ws.y, s[1], t);
          t = fmaf(ws.z, s[2], t);
          t = fmaf(ws.w, s[3], t);
          acc[cl] = t;
        }
      }
    }
  }
}

// Features at d = 32 and 64 (one or two lanes per vector): a lane's 16-byte
// pieces of one row are 2 E d floats away from its neighbours' rows, so the
// warp first lays its VPW rows of cos and of sin out in shared memory (row
// stride d + 4T words: conflict-free for the 128-bit stores of layout A) and
// then writes them back row by row, each instruction covering 512 contiguous
// bytes of one or more rows (128-byte segments at d = 32).
constexpr int kRowsBuf = 2 * 1152;  // cos and sin rows: 2 x VPW (d + 4T) floats

template <int L>
__device__ __forceinline__ void epilogue_rows(const Launch& P, int64_t n0, int e, int g, int lam,
                                              const float (&h)[32], const float (&cs)[32],
                                              float* buf) {
  using Y = Lay<L>;
  constexpr int d = Y::d, RS = d + 4 * Y::T, HALF = (32 / Y::T) * RS;
  static_assert(2 * HALF <= kRowsBuf, "row buffer");
  const int lane = threadIdx.x & 31;
  const int64_t F = 2ll * P.a.E * d;
  __syncwarp();  // every lane is done with the buffer's previous contents
#pragma unroll
  for (int m = 0; m < 8; ++m) {
    float c[4], s4[4];
    cos_sin4(&cs[4 * m], &h[4 * m], c, s4);
    const int at = g * RS + Y::kA(lam, 4 * m);
    *reinterpret_cast<float4*>(buf + at) = make_float4(c[0], c[1], c[2], c[3]);
    *reinterpret_cast<float4*>(buf + HALF + at) = make_float4(s4[0], s4[1], s4[2], s4[3]);
  }
  __syncwarp();
#pragma unroll
  for (int i = 0; i < 8; ++i) {
    const int f = 128 * i + 4 * lane;  // element of the warp's VPW x d block
    const int r = f / d, col = f % d;
    const int64_t n = n0 + r;
    if (n < P.a.n) {
      float* o = P.phi + n * F + 2ll * e * d + col;
      __stcs(reinterpret_cast<float4*>(o), *reinterpret_cast<const float4*>(buf + r * RS + col));
      __stcs(reinterpret_cast<float4*>(o + d),
             *reinterpret_cast<const float4*>(buf + HALF + r * RS + col));
    }
  }
  __syncwarp();  // the rows are read before the buffer is reused
}

// ---------------------------------------------------------------------------
// Warp kernel, 5 <= L <= 10.
// ---------------------------------------------------------------------------
// Work item = (tile of SPI samples, expansion). Small tiles keep a warp's
// input rows resident in L1 while it walks the expansions of its tile; the
// cost is one table load per item, which the lane-ordered tables keep to a
// few coalesced loads.
template <int L>
struct WarpShape {
  static constexpr int T = Lay<L>::T;
  static constexpr int VPW = 32 / T;                 // samples per warp step
  static constexpr int R = VPW >= 4 ? 1 : 4 / VPW;   // steps per item
  static constexpr int SPI = VPW * R;                // samples per item
};

template <int L, int MODE, bool ONE = false>
__global__ void __launch_bounds__(kWarps * 32, MODE == MODE_FEATURES ? kWarpMinBlocks : 12) k_feat_warp(const Launch P) {
  using Y = Lay<L>;
  using WS = WarpShape<L>;
  constexpr int d = Y::d;
  // Row-wise output stores at d = 32 and 64 (feature sweep: 0.746 -> 0.337 ms
  // and 0.409 -> 0.381 ms); at d = 128 the staging cost more than it saved.
  constexpr bool kRows = MODE == MODE_FEATURES && L <= 6;
  // At d = 32 a lane holds a whole vector and the slot serves only u and the
  // Pi gather (the layout moves are identities there): an odd stride puts the
  // 32 vectors' slots on 32 distinct banks for both the stores and the gather
  // (every vector of the warp gathers the same positions), instead of 4-way
  // conflicts with the padded stride.
  constexpr int kSlot = L == 5 ? 33 : Y::SLOT;
  constexpr int kBuf = kRows && kRowsBuf > WS::VPW * kSlot ? kRowsBuf : WS::VPW * kSlot;
  __shared__ __align__(16) float sm[kWarps][kBuf];
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int g = lane / Y::T, lam = lane % Y::T;
  float* buf = sm[warp];
  const uint32_t buf_addr = smem_addr(buf);

  const int E = P.a.E;
  // Tiles of R rounds of VPW samples; ONE (a small batch: fewer full tiles
  // than resident warps) runs one round per tile, so that more warps share it.
  constexpr int R = ONE ? 1 : WS::R;
  constexpr int spi = WS::VPW * R;
  const int64_t tiles = (P.a.n + spi - 1) / spi;
  const int64_t items = tiles * E;
  const int64_t nw = (int64_t)gridDim.x * kWarps;
  const int64_t wid = (int64_t)blockIdx.x * kWarps + warp;
  const int64_t it0 = items * wid / nw, it1 = items * (wid + 1) / nw;

  uint32_t bmask = 0;
  float gt[32], cs[32];
  uint32_t poff[16];  // gather byte offsets inside the slot, two 16-bit values each
  uint32_t pslot = 0;
  uint32_t ubase = 0;  // d = 1024: this lane's word base in the skewed slot
  int cur_e = -1;

  for (int64_t it = it0; it < it1; ++it) {
    // Features: expansion fastest (x rows of a tile reused from L1 across e).
    // Logits: tile fastest (the expansion's slice of W stays in L1).
    int64_t tile;
    int e;
    if constexpr (MODE == MODE_FEATURES) {
      tile = it / E;
      e = (int)(it % E);
    } else {
      e = (int)(it / tiles);
      tile = it % tiles;
    }
    if (e != cur_e) {
      cur_e = e;
      const int64_t off = (int64_t)e * d;
      // Lane-ordered tables: entry (m, lam, q) holds element kB(lam, 4m+q).
      bmask = __ldg(P.a.maskA + (int64_t)e * Y::T + lam);
      const uint32_t slot = buf_addr + 4u * (uint32_t)(g * kSlot);
      // Gather offsets are below 2^16 bytes: two per register.
      pslot = slot;
      if constexpr (L == 10) {  // skewed slot, offsets packed at plan time
        ubase = __ldg(P.a.ubase + (int64_t)e * 32 + lam);
        load_skew_offsets(P.a.permS + (int64_t)e * (d / 2), lam, poff);
      } else {
        const uint4* pb = reinterpret_cast<const uint4*>(P.a.permB + off) + lam;
#pragma unroll
        for (int m = 0; m < 8; ++m) {
          const uint4 v = __ldg(pb + m * Y::T);
          poff[2 * m] = v.x | (v.y << 16);
          poff[2 * m + 1] = v.z | (v.w << 16);
        }
      }
      if (P.a.GB) {
        const float4* gb = reinterpret_cast<const float4*>(P.a.GB + off) + lam;
#pragma unroll
        for (int m = 0; m < 8; ++m) {
          const float4 v = __ldg(gb + m * Y::T);
          gt[4 * m] = v.x;
          gt[4 * m + 1] = v.y;
          gt[4 * m + 2] = v.z;
          gt[4 * m + 3] = v.w;
        }
      } else {  // caller-supplied G, natural order
#pragma unroll
        for (int j = 0; j < 32; ++j) gt[j] = __ldg(P.a.G + off + Y::kB(lam, j));
      }
#pragma unroll
      for (int m = 0; m < 8; ++m) {
        const float4 v = __ldg(reinterpret_cast<const float4*>(P.a.Cs + off + Y::kA(lam, 4 * m)));
        cs[4 * m] = v.x;
        cs[4 * m + 1] = v.y;
        cs[4 * m + 2] = v.z;
        cs[4 * m + 3] = v.w;
      }
    }
    for (int r = 0; r < R; ++r) {
      const int64_t n = tile * spi + r * WS::VPW + g;
      const bool valid = n < P.a.n;
      float w[32];
      load_x_A<L>(P, n, valid, lam, w);
      // Ask L1 for the next sample's row now; it is needed one sample later.
      {
        int64_t nn;
        bool more = true;
        if (r + 1 < R) {
          nn = n + WS::VPW;
        } else {
          const int64_t it2 = it + 1;
          more = it2 < it1;
          const int64_t tile2 = (MODE == MODE_FEATURES) ? it2 / E : it2 % tiles;
          nn = tile2 * spi + g;
        }
        if (more && nn < P.a.n && (int64_t)lam * 32 < P.a.in_dim)
          asm volatile("prefetch.global.L1 [%0];" ::"l"(P.a.x + nn * P.a.ldx + lam * 32));
      }
      apply_signs(w, bmask);
      // u = H B x-hat
      hreg<Y::maskA()>(w);
      if constexpr (L > 5) {
        store_A<L>(buf, g, lam, w);
        __syncwarp();
        load_B<L>(buf, g, lam, w);
      }
      hreg<Y::maskB()>(w);
      // v = Pi u: u goes to shared memory, each register gathers its source.
      if constexpr (L == 10) {
        store_skew(buf, ubase, w);
      } else if constexpr (L == 5) {
        float* q = buf + g * kSlot;
#pragma unroll
        for (int j = 0; j < 32; ++j) q[j] = w[j];
      } else {
        store_B<L>(buf, g, lam, w);
      }
      __syncwarp();
#pragma unroll
      for (int j = 0; j < 32; ++j)
        w[j] = lds32(pslot + ((j & 1) ? (poff[j >> 1] >> 16) : (poff[j >> 1] & 0xffffu)));
      // h = H G v (G folded into the first butterfly stage)
      hreg_scaled<Y::maskB()>(w, gt);
      if constexpr (L > 5) {
        __syncwarp();  // every lane finished gathering before the slots are reused
        store_B<L>(buf, g, lam, w);
        __syncwarp();
        load_A<L>(buf, g, lam, w);
      }
      hreg<Y::maskA()>(w);
      float acc[CMAX];
#pragma unroll
      for (int c = 0; c < CMAX; ++c) acc[c] = 0.f;
      if constexpr (kRows)
        epilogue_rows<L>(P, n - g, e, g, lam, w, cs, buf);
      else
        epilogue_A<L, MODE>(P, n, e, valid, lam, w, cs, acc);
      if constexpr (MODE == MODE_LOGITS) {
#pragma unroll
        for (int c = 0; c < CMAX; ++c) {
          float t = acc[c];
#pragma unroll
          for (int o = Y::T / 2; o > 0; o >>= 1) t += __shfl_xor_sync(0xffffffffu, t, o);
          acc[c] = t;
        }
        if (valid && lam == 0) {
          float* pr = P.part + (n * E + e) * P.C;
#pragma unroll
          for (int c = 0; c < CMAX; ++c)
            if (c < P.C) pr[c] = acc[c];
        }
      }
      if constexpr (L == 5) __syncwarp();
    }
  }
}

// ---------------------------------------------------------------------------
// Block kernel, 11 <= L <= 15: one block of T = 2^(L-5) threads per (n, e).
// ---------------------------------------------------------------------------
template <int L, int MODE>
__global__ void __launch_bounds__(1 << (L - 5)) k_feat_cta(const Launch P) {
  using Y = Lay<L>;
  constexpr int d = Y::d, T = Y::T, NWARP = T / 32;
  extern __shared__ float4 sm4[];
  float* buf = reinterpret_cast<float*>(sm4);
  __shared__ float red[NWARP][CMAX];
  const uint32_t buf_addr = smem_addr(buf);
  const int lam = threadIdx.x;
  const int E = P.a.E;
  const int64_t items = P.a.n * E;
  for (int64_t it = blockIdx.x; it < items; it += gridDim.x) {
    const int64_t n = it / E;
    const int e = (int)(it % E);
    const int64_t off = (int64_t)e * d;
    float w[32];
    load_x_A<L>(P, n, true, lam, w);
    apply_signs(w, load_bmask_A<L>(P.a.B_bits + (int64_t)e * (d / 32), lam));
    hreg<Y::maskA()>(w);
    store_A<L>(buf, 0, lam, w);
    __syncthreads();
    if constexpr (L == 15) {
      // The next item's row into L2 (4 KB per warp) when it is another row,
      // issued after this item's loads: features at 2^15 0.479 -> 0.459 ms.
      const int64_t n2 = (it + gridDim.x) / E;
      const int64_t lo = (int64_t)(lam >> 5) * 1024;
      if (P.vec_x && it + gridDim.x < items && n2 != n && (lam & 31) == 0 && lo < P.a.in_dim) {
        const int64_t cnt = P.a.in_dim - lo < 1024 ? (P.a.in_dim - lo) & ~int64_t(3) : 1024;
        if (cnt > 0) prefetch_l2_bulk(P.a.x + n2 * P.a.ldx + lo, (uint32_t)(4 * cnt));
      }
    }
    load_B<L>(buf, 0, lam, w);
    hreg<Y::maskB()>(w);
    store_B<L>(buf, 0, lam, w);
    __syncthreads();
    load_C<L>(buf, lam, w);
    hreg<Y::maskC()>(w);
    store_C<L>(buf, lam, w);
    __syncthreads();
    // gather into layout C, then G and the C-phase of the second transform
    float gt[32];
#pragma unroll
    for (int j = 0; j < 32; ++j) {
      const int k = Y::kC(lam, j);
      const uint32_t src = __ldg(P.a.perm + off + k);
      gt[j] = __ldg(P.a.G + off + k);
      w[j] = lds32(buf_addr + 4u * (uint32_t)spos<L>(0, (int)src));
    }
    hreg_scaled<Y::maskC()>(w, gt);
    __syncthreads();
    store_C<L>(buf, lam, w);
    __syncthreads();
    load_B<L>(buf, 0, lam, w);
    hreg<Y::maskB()>(w);
    store_B<L>(buf, 0, lam, w);
    __syncthreads();
    load_A<L>(buf, 0, lam, w);
    hreg<Y::maskA()>(w);
    float cs[32];
#pragma unroll
    for (int m = 0; m < 8; ++m) {
      const float4 v = __ldg(reinterpret_cast<const float4*>(P.a.Cs + off + Y::kA(lam, 4 * m)));
      cs[4 * m] = v.x;
      cs[4 * m + 1] = v.y;
      cs[4 * m + 2] = v.z;
      cs[4 * m + 3] = v.w;
    }
    float acc[CMAX];
#pragma unroll
    for (int c = 0; c < CMAX; ++c) acc[c] = 0.f;
    epilogue_A<L, MODE>(P, n, e, true, lam, w, cs, acc);
    if constexpr (MODE == MODE_LOGITS) {
#pragma unroll
      for (int c = 0; c < CMAX; ++c) {
        float t = acc[c];
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) t += __shfl_xor_sync(0xffffffffu, t, o);
        if ((lam & 31) == 0) red[lam >> 5][c] = t;
      }
      __syncthreads();
      if (lam < P.C) {
        float t = 0.f;
        for (int q = 0; q < NWARP; ++q) t += red[q][lam];
        P.part[(n * E + e) * P.C + lam] = t;
      }
    }
    __syncthreads();
  }
}

// ---------------------------------------------------------------------------
// Thread kernel, 1 <= L <= 4: one thread per (n, e), everything in registers.
// ---------------------------------------------------------------------------
template <int L>
__device__ __forceinline__ void hsmall(float (&w)[1 << L]) {
#pragma unroll
  for (int h = 1; h < (1 << L); h <<= 1)
#pragma unroll
    for (int k = 0; k < (1 << L); ++k)
      if (!(k & h)) {
        const float a = w[k], c = w[k | h];
        w[k] = a + c;
        w[k | h] = a - c;
      }
}

template <int L, int MODE>
__global__ void __launch_bounds__(128) k_feat_tiny(const Launch P) {
  constexpr int d = 1 << L;
  const int E = P.a.E;
  const int64_t items = P.a.n * E;
  const int64_t F = 2ll * E * d;
  for (int64_t it = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; it < items;
       it += (int64_t)gridDim.x * blockDim.x) {
    const int64_t n = it / E;
    const int e = (int)(it % E);
    const int64_t off = (int64_t)e * d;
    const float* row = P.a.x + n * P.a.ldx;
    const uint32_t bits = __ldg(P.a.B_bits + e);
    float u[d], w[d];
#pragma unroll
    for (int k = 0; k < d; ++k) {
      const float xv = (k < P.a.in_dim) ? __ldg(row + k) : 0.f;
      u[k] = (bits >> k & 1u) ? -xv : xv;
    }
    hsmall<L>(u);
#pragma unroll
    for (int k = 0; k < d; ++k) {
      const uint32_t src = __ldg(P.a.perm + off + k);
      float v = 0.f;
#pragma unroll
      for (int q = 0; q < d; ++q) v = (src == (uint32_t)q) ? u[q] : v;  // register select, no local memory
      w[k] = __ldg(P.a.G + off + k) * v;
    }
    hsmall<L>(w);
    float acc[CMAX];
#pragma unroll
    for (int c = 0; c < CMAX; ++c) acc[c] = 0.f;
#pragma unroll
    for (int k = 0; k < d; ++k) {
      float c, s;
      cos_sin(__ldg(P.a.Cs + off + k) * w[k], c, s);
      if constexpr (MODE == MODE_FEATURES) {
        P.phi[n * F + 2ll * e * d + k] = c;
        P.phi[n * F + 2ll * e * d + d + k] = s;
      } else {
        for (int cl = 0; cl < P.C; ++cl) {
          const float* wr = P.W + cl * F + 2ll * e * d;
          acc[cl] = fmaf(__ldg(wr + k), c, fmaf(__ldg(wr + d + k), s, acc[cl]));
        }
      }
    }
    if constexpr (MODE == MODE_LOGITS) {
      for (int cl = 0; cl < P.C; ++cl) P.part[(n * E + e) * P.C + cl] = acc[cl];
    }
  }
}

// logits[n][c] = b[c] + sum_e part[n][e][c], expansions summed in order.
__global__ void k_logits_reduce(const float* __restrict__ part, const float* __restrict__ b,
                                int64_t n, int E, int C, float* __restrict__ logits) {
  const int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= n * C) return;
  const int64_t i = t / C;
  const int c = (int)(t % C);
  float s = 0.f;
  for (int e = 0; e < E; ++e) s += part[(i * E + e) * C + c];
  logits[t] = s + (b ? b[c] : 0.f);
}

// ---------------------------------------------------------------------------
// Fused logits at d = 1024, warp-specialised. A block of 16 warps owns tiles
// of 8 rows. Warps 0..7 produce: for each (tile, expansion e) warp w computes
// the 2048 features of row w (the feature kernel's sequence) into its 8 KB
// slice of one of two shared 8 x 2048 phi buffers; the slice is also the
// warp's transpose buffer while the transforms run. Warps 8..15 consume: they
// contract the buffer with W_e while the producers fill the other one. The
// buffers change hands on named barriers (FULL: producers arrive, consumers
// wait; EMPTY: the reverse). Consumer thread (class group cg, feature thread
// ft) owns classes [cg*CPT, cg*CPT + CPT) and float4 columns ft, ft + TPG, ...
// of all 8 rows, so each weight is loaded once per 8 rows, one column ahead of
// its use; its 8 x CPT partial sums stay in registers for the whole tile and
// are reduced once per tile in a fixed order.
// ---------------------------------------------------------------------------
constexpr int kTileRows = 8;
constexpr int kTileWarps = 2 * kTileRows;

// Chunks of expansions per tile: 1 while the tiles alone fill the SMs, else
// as many as keep one block per SM busy (a batch of 512 rows has 64 tiles).
int logits_echunks(int64_t n, int E, int num_sms) {
  const int64_t tiles = (n + kTileRows - 1) / kTileRows;
  if (tiles >= num_sms) return 1;
  const int64_t c = num_sms / tiles;
  return (int)std::max<int64_t>(1, std::min<int64_t>(c, E));
}
constexpr int kTileThreads = kTileWarps * 32;
constexpr int kConsumers = kTileRows * 32;
constexpr int kBarFull = 1, kBarEmpty = 3, kBarReduce = 5;  // ids 1-2, 3-4, 5

// One float4 column of CPT weight rows. W streams through once per tile: the
// loads skip L1 so that the producers' tables and rows stay there.
template <int CPT, int CG>
__device__ __forceinline__ void load_w_col(const float* __restrict__ Wg, int64_t F, int C, int cg,
                                           int f4, float4 (&w)[CPT]) {
#pragma unroll
  for (int c = 0; c < CPT; ++c) {
    w[c] = make_float4(0.f, 0.f, 0.f, 0.f);
    if (cg * CPT + c < C) {
      const float4* q = reinterpret_cast<const float4*>(Wg + c * F) + f4;
      asm("ld.global.nc.L1::no_allocate.v4.f32 {%0, %1, %2, %3}, [%4];"
          : "=f"(w[c].x), "=f"(w[c].y), "=f"(w[c].z), "=f"(w[c].w)
          : "l"(q));
    }
  }
}

// x = hi + lo + O(2^-22 x) with hi, lo fp16 (pairs packed as half2).
__device__ __forceinline__ void split_f16(float a, float b, uint32_t& hi, uint32_t& lo) {
  const __half2 h = __floats2half2_rn(a, b);
  const float2 hf = __half22float2(h);
  const __half2 l = __floats2half2_rn(a - hf.x, b - hf.y);  // both differences are exact
  hi = *reinterpret_cast<const uint32_t*>(&h);
  lo = *reinterpret_cast<const uint32_t*>(&l);
}

// One row-expansion of a fused-logits producer at d = 1024: the features of
// sample n under expansion e (zeros for an invalid row) into the row slice
// buf (also the transform's shared slot), cos then sin, FP32 in natural order
// (buf[0, 2048)). The feature kernel's sequence: signs, H over layouts A and
// B, u into the skewed slot, the Pi gather, G, H, z = Cs h.
__device__ __forceinline__ void produce_row_1024(const Launch& P, int64_t n, bool valid, int e,
                                                 int lane, float* buf) {
  constexpr int L = 10;
  using Y = Lay<L>;
  constexpr int d = Y::d;
  const uint32_t slot = smem_addr(buf);
  const int64_t off = (int64_t)e * d;
  const uint32_t bmask = __ldg(P.a.maskA + (int64_t)e * Y::T + lane);
  const uint32_t ubase = __ldg(P.a.ubase + (int64_t)e * 32 + lane);
  uint32_t poff[16];
  float gt[32];
  load_skew_offsets(P.a.permS + (int64_t)e * (d / 2), lane, poff);
  if (P.a.GB) {
    const float4* gb = reinterpret_cast<const float4*>(P.a.GB + off) + lane;
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
    for (int j = 0; j < 32; ++j) gt[j] = __ldg(P.a.G + off + Y::kB(lane, j));
  }
  float w[32];
  load_x_A<L>(P, n, valid, lane, w);
  apply_signs(w, bmask);
  hreg<Y::maskA()>(w);
  store_A<L>(buf, 0, lane, w);
  __syncwarp();
  load_B<L>(buf, 0, lane, w);
  hreg<Y::maskB()>(w);
  store_skew(buf, ubase, w);
  __syncwarp();
#pragma unroll
  for (int j = 0; j < 32; ++j)
    w[j] = lds32(slot + ((j & 1) ? (poff[j >> 1] >> 16) : (poff[j >> 1] & 0xffffu)));
  hreg_scaled<Y::maskB()>(w, gt);
  __syncwarp();
  store_B<L>(buf, 0, lane, w);
  __syncwarp();
  load_A<L>(buf, 0, lane, w);
  hreg<Y::maskA()>(w);
  __syncwarp();  // every lane holds its values: the slice takes the features now
#pragma unroll
  for (int m = 0; m < 8; ++m) {
    const int k0 = Y::kA(lane, 4 * m);
    const float4 c4 = __ldg(reinterpret_cast<const float4*>(P.a.Cs + off + k0));
    const float cs[4] = {c4.x, c4.y, c4.z, c4.w};
    float c[4], s4[4];
    cos_sin4(cs, &w[4 * m], c, s4);
    // an invalid row contributes nothing
    if (!valid) c[0] = c[1] = c[2] = c[3] = s4[0] = s4[1] = s4[2] = s4[3] = 0.f;
    *reinterpret_cast<float4*>(buf + k0) = make_float4(c[0], c[1], c[2], c[3]);
    *reinterpret_cast<float4*>(buf + d + k0) = make_float4(s4[0], s4[1], s4[2], s4[3]);
  }
}

template <int CPT, int CG>
__global__ void __launch_bounds__(kTileThreads, 1) k_logits_tile(const Launch P,
                                                                 const float* __restrict__ b,
                                                                 float* __restrict__ logits,
                                                                 int echunks) {
  constexpr int L = 10;
  using Y = Lay<L>;
  constexpr int d = Y::d, F2 = 2 * d, F24 = F2 / 4;
  constexpr int TPG = kConsumers / CG;  // consumer threads per class group
  constexpr int ITER = F24 / TPG;       // float4 columns per consumer thread and expansion
  static_assert(Y::SLOT <= F2 && F24 % TPG == 0 && TPG % 32 == 0, "tile shape");
  static_assert(kTileRows * 10 == (d / 2 + 2 * d) / 32, "8 producer warps x 10 lines cover permS, G and Cs");
  extern __shared__ float4 sm4[];
  float* phis = reinterpret_cast<float*>(sm4);  // [2][kTileRows][F2]
  float* red = phis + 2 * kTileRows * F2;       // [8 consumer warps][kTileRows][CPT]
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int C = P.C, E = P.a.E;
  const int64_t F = 2ll * E * d;
  // Work units: (tile, chunk of expansions); with echunks > 1 a unit writes
  // its partial logits (no bias) for a later fixed-order sum over chunks.
  const int64_t tiles = (P.a.n + kTileRows - 1) / kTileRows;
  const int64_t units = tiles * echunks;
  if (warp < kTileRows) {
    // ------------------------------ producers ------------------------------
    int64_t step = 0;
    for (int64_t u = blockIdx.x; u < units; u += gridDim.x) {
      const int64_t tile = u / echunks;
      const int ch = (int)(u % echunks);
      const int e0 = E * ch / echunks, e1 = E * (ch + 1) / echunks;
      const int64_t n = tile * kTileRows + warp;
      const bool valid = n < P.a.n;
      for (int e = e0; e < e1; ++e, ++step) {
        const int bsel = (int)(step & 1);
        if (step >= 2) named_barrier(kBarEmpty + bsel, kTileThreads);
        float* buf = phis + (bsel * kTileRows + warp) * F2;
        {  // the next step's tables (permS, G, Cs: 80 lines of 128 B) into L1, 10 per warp
          const int64_t offn = (int64_t)(e + 1 < E ? e + 1 : 0) * d;
          if (lane < 10) {
            const int li = warp * 10 + lane;
            const float* gsrc = P.a.GB ? P.a.GB : P.a.G;
            const char* line =
                li < 16   ? reinterpret_cast<const char*>(P.a.permS + offn / 2) + li * 128
                : li < 48 ? reinterpret_cast<const char*>(gsrc + offn) + (li - 16) * 128
                          : reinterpret_cast<const char*>(P.a.Cs + offn) + (li - 48) * 128;
            asm volatile("prefetch.global.L1 [%0];" ::"l"(line));
          }
        }
        produce_row_1024(P, n, valid, e, lane, buf);
        named_arrive(kBarFull + bsel, kTileThreads);
      }
    }
    // Wait out the consumers' last two releases so every arrival is matched.
    for (int64_t s = step < 2 ? 2 : step; s < step + 2; ++s)
      named_barrier(kBarEmpty + (int)(s & 1), kTileThreads);
    return;
  }
  // ------------------------------- consumers -------------------------------
  const int ct = threadIdx.x - kConsumers, cw = ct >> 5;
  const int cg = ct / TPG, ft = ct % TPG;
  const float* Wc = P.W + (int64_t)(cg * CPT) * F;
  // Up to 5 classes per thread the next column's weights are loaded one column
  // ahead (2 x 5 float4 registers); with more, at their use, to avoid spills.
  constexpr bool kAhead = CPT <= 5;
  int64_t step = 0;
  float4 wn[CPT];
  if (kAhead && blockIdx.x < units) {
    const int ch = (int)(blockIdx.x % echunks);
    load_w_col<CPT, CG>(Wc + 2ll * (E * ch / echunks) * d, F, C, cg, ft, wn);
  }
  for (int64_t u = blockIdx.x; u < units; u += gridDim.x) {
    const int64_t tile = u / echunks;
    const int ch = (int)(u % echunks);
    const int e0 = E * ch / echunks, e1 = E * (ch + 1) / echunks;
    float acc[kTileRows * CPT];
#pragma unroll
    for (int i = 0; i < kTileRows * CPT; ++i) acc[i] = 0.f;
    for (int e = e0; e < e1; ++e, ++step) {
      const int bsel = (int)(step & 1);
      const float4* ph4 = reinterpret_cast<const float4*>(phis + bsel * kTileRows * F2);
      const float* Wg = Wc + 2ll * e * d;
      named_barrier(kBarFull + bsel, kTileThreads);
#pragma unroll
      for (int it = 0; it < ITER; ++it) {
        float4 wv[CPT];
        if constexpr (kAhead) {
#pragma unroll
          for (int c = 0; c < CPT; ++c) wv[c] = wn[c];
          // the next column: this expansion's, else the next step's first
          if (it + 1 < ITER) {
            load_w_col<CPT, CG>(Wg, F, C, cg, ft + (it + 1) * TPG, wn);
          } else {
            int en = e + 1;
            bool more = en < e1;
            if (!more && u + gridDim.x < units) {
              more = true;
              en = E * (int)((u + gridDim.x) % echunks) / echunks;
            }
            if (more) load_w_col<CPT, CG>(Wc + 2ll * en * d, F, C, cg, ft, wn);
          }
        } else {
          load_w_col<CPT, CG>(Wg, F, C, cg, ft + it * TPG, wv);
        }
        const int f4 = ft + it * TPG;
#pragma unroll
        for (int s = 0; s < kTileRows; ++s) {
          const float4 p = ph4[s * F24 + f4];
#pragma unroll
          for (int c = 0; c < CPT; ++c) {
            float t = acc[s * CPT + c];
            t = fmaf(wv[c].x, p.x, t);
            t = fmaf(wv[c].y, p.y, t);
            t = fmaf(wv[c].z, p.z, t);
            acc[s * CPT + c] = fmaf(wv[c].w, p.w, t);
          }
        }
      }
      named_arrive(kBarEmpty + bsel, kTileThreads);
    }
    // ---- reduce over the TPG threads of each class group (fixed order) ----
#pragma unroll
    for (int i = 0; i < kTileRows * CPT; ++i) {
      float t = acc[i];
#pragma unroll
      for (int o = 16; o > 0; o >>= 1) t += __shfl_xor_sync(0xffffffffu, t, o);
      acc[i] = t;
    }
    if (lane == 0) {
#pragma unroll
      for (int i = 0; i < kTileRows * CPT; ++i) red[cw * kTileRows * CPT + i] = acc[i];
    }
    named_barrier(kBarReduce, kConsumers);
    constexpr int wpg = TPG / 32;  // consumer warps per class group
    for (int o = ct; o < kTileRows * C; o += kConsumers) {
      const int s = o / C, cls = o % C;
      const int g2 = cls / CPT, c = cls % CPT;
      float t = 0.f;
      for (int q = 0; q < wpg; ++q) t += red[(g2 * wpg + q) * kTileRows * CPT + s * CPT + c];
      const int64_t row = tile * kTileRows + s;
      if (row < P.a.n) {
        if (echunks == 1) logits[row * C + cls] = t + (b ? b[cls] : 0.f);
        else P.part[(row * echunks + ch) * C + cls] = t;
      }
    }
    named_barrier(kBarReduce, kConsumers);  // red is free for the next tile
  }
}

template <int CPT, int CG>
cudaError_t run_logits_tile(const Launch& P, const float* b, float* logits, cudaStream_t s) {
  using Y = Lay<10>;
  const size_t smem = sizeof(float) * (2 * kTileRows * 2 * Y::d + kTileRows * kTileRows * CPT);
  cudaError_t err = cudaFuncSetAttribute(k_logits_tile<CPT, CG>,
                                         cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (err != cudaSuccess) return err;
  const int echunks = logits_echunks(P.a.n, P.a.E, P.a.num_sms);
  const int64_t units = (P.a.n + kTileRows - 1) / kTileRows * echunks;
  const unsigned grid =
      (unsigned)std::max<int64_t>(1, std::min<int64_t>(units, (int64_t)P.a.num_sms));
  k_logits_tile<CPT, CG><<<grid, kTileThreads, smem, s>>>(P, b, logits, echunks);
  err = cudaGetLastError();
  if (err != cudaSuccess || echunks == 1) return err;
  const int64_t total = P.a.n * P.C;
  k_logits_reduce<<<(unsigned)((total + 255) / 256), 256, 0, s>>>(P.part, b, P.a.n, echunks, P.C,
                                                                  logits);
  return cudaGetLastError();
}

// ---------------------------------------------------------------------------
// Fused logits at d = 1024 with the contraction W phi on the tensor cores.
// Blocks of kMmaWarps warps own tiles of 16 rows (the M of mma.m16n8k16),
// several blocks per SM, and every warp takes both roles in turn. Per
// expansion: warp w loads the expansion's tables into registers once and
// computes, for its rows w, w + kMmaWarps, ... of the tile, the FP32
// sequence of k_feat_warp up to the phases z = Cs h (in the row's slice of
// the shared buffer, which is also its transform slot), and writes z there.
// After a block barrier, warp w contracts the features of its z positions
// (1024 / kMmaWarps of them) over all 16 rows: for each pair of k-steps (the
// cos features of 16 positions and the sin features of the same positions,
// k-steps ks and ks + 64) a lane reads the z of its fragment positions,
// forms cos z and sin z (the arithmetic of the feature kernel, bit for bit),
// splits each into fp16 hi = round(x), lo = round(x - hi) as A fragments,
// and takes W as the B operand, split the same way ahead of the launch
// (k_logits_wsplit) after scaling class c by a power of two 2^s_c (exact),
// which keeps every class's weights inside fp16's range. The products of a
// pair, lo.hi + hi.lo + hi.hi for each of its two k-steps (the lo.lo term is
// below 2^-22 of the product), go into a fresh FP32 accumulator that is then
// added to the running sum with a rounded FP32 add: the tensor core's own
// accumulation truncates relative to the running value, which over hundreds
// of steps into one accumulator left errors of 1e-4 on logits of a few
// units. The running sums live in a per-lane slice of shared memory across
// the expansions, which leaves the producer its registers for the tables. A
// second block barrier frees the buffer for the next expansion. After the
// last expansion of a tile the warps' sums are added in a fixed order and
// scaled back by 2^-s_c. The blocks of an SM drift out of phase, so one
// block's contraction (its cos and sin on the special-function units, its
// MMAs) overlaps another's production (FP32 butterflies, shared memory).
//
// Measured at 60000 rows, E = 16, 10 classes, on one GPU: three 4-warp
// blocks per SM (four rows per warp and table load, up to 170 registers)
// 2.24 ms (E = 8: 1.14 ms); two 8-warp blocks 2.27 ms (1.16 ms), the same
// with Cs also held across the rows (it spills) 2.33 ms. One 16-warp block
// per SM with 32-row tiles: 2.67 ms (1.35 ms; production alone 1.76 ms, the contraction alone
// 1.12 ms: the two phases of one block do not overlap). With the split
// features (twice the bytes of z) in a 16-row buffer and one row per warp
// and expansion: 2.82 ms (1.44 ms); as dedicated roles (12 producer warps
// filling double-buffered 12-row tiles for 4 contracting warps that stream
// W through a register ring) 2.87 ms; transposed (classes as M, 8-row tiles
// as N, two 8-warp blocks per SM) 2.85 ms. Storing z rather than the
// features halves the buffer, which lets a warp produce several rows per
// load of the expansion's tables and leaves room for several blocks per SM.
// ---------------------------------------------------------------------------
constexpr int kMmaWarps = 4;
constexpr int kMmaBlocksPerSM = 3;
constexpr int kMmaThreads = kMmaWarps * 32;
constexpr int kMmaRows = 16;                     // rows per tile
constexpr int kMmaRPW = kMmaRows / kMmaWarps;    // rows per warp and table load
constexpr int kMmaMT = kMmaRows / 16;            // M tiles per tile
constexpr int kMmaKP = 64 / kMmaWarps;           // (cos, sin) k-step pairs per warp
constexpr int kMmaZS = 1024 + 40;                // words per z row: >= the transform slot, = 8 mod 32
constexpr int kMmaAccS = 4 * (2 * kMmaMT + 1);   // words per lane of the running sums (8 MT used)
constexpr int kMmaKsteps = 2 * 1024 / 16;        // 16-feature k-steps per expansion
constexpr int kMmaPrefetchLines = 80 / kMmaWarps;  // the 80 table lines per expansion

int logits_mma_echunks(int64_t n, int E, int num_sms) {
  const int64_t tiles = (n + kMmaRows - 1) / kMmaRows;
  const int64_t slots = (int64_t)num_sms * kMmaBlocksPerSM;
  if (tiles >= slots) return 1;
  const int64_t c = slots / tiles;
  return (int)std::max<int64_t>(1, std::min<int64_t>(c, E));
}

// B fragments of W (C x 2Ed) for the tensor-core logits. Block c fills class
// slot c of the fragments (8 NT slots; zeros past C): with g = c % 8 and
// nt = c / 8, lane 4 g + t of k-step ks of expansion e holds, as fp16 hi/lo
// pairs, W_c at features 16 ks + 2 t, +1 (register b0) and 16 ks + 2 t + 8, +9
// (b1) of the expansion, after scaling the class by 2^s_c with its largest
// magnitude in [2^14, 2^15); inv[c] = 2^-s_c.
template <int NT>
__global__ void __launch_bounds__(256) k_logits_wsplit(const float* __restrict__ W, int C, int E,
                                                       uint4* __restrict__ wf,
                                                       float* __restrict__ inv) {
  const int cls = blockIdx.x, g = cls & 7, nt = cls >> 3;
  const int64_t F = 2ll * E * 1024;
  const float* wr = W + (int64_t)cls * F;
  const bool valid = cls < C;
  __shared__ float wmax[8];
  float m = 0.f;
  if (valid)
    for (int64_t k = threadIdx.x; k < F; k += blockDim.x) m = fmaxf(m, fabsf(__ldg(wr + k)));
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) m = fmaxf(m, __shfl_xor_sync(0xffffffffu, m, o));
  if ((threadIdx.x & 31) == 0) wmax[threadIdx.x >> 5] = m;
  __syncthreads();
  m = 0.f;
#pragma unroll
  for (int i = 0; i < 8; ++i) m = fmaxf(m, wmax[i]);
  int se = 0;  // scale exponent: m 2^se in [2^14, 2^15)
  if (m > 0.f) se = min(max(14 - (((__float_as_int(m) >> 23) & 0xff) - 127), -100), 100);
  const float scale = __int_as_float((se + 127) << 23);
  if (threadIdx.x == 0 && valid) inv[cls] = __int_as_float((127 - se) << 23);
  const int items = E * kMmaKsteps * 4;  // (expansion, k-step, t)
  for (int it = threadIdx.x; it < items; it += blockDim.x) {
    const int t = it & 3;
    const int eks = it >> 2;  // e * kMmaKsteps + ks
    uint4 v = make_uint4(0u, 0u, 0u, 0u);
    if (valid) {
      const int e = eks / kMmaKsteps, ks = eks % kMmaKsteps;
      const float* q = wr + (int64_t)e * 2048 + 16 * ks + 2 * t;
      split_f16(__ldg(q) * scale, __ldg(q + 1) * scale, v.x, v.z);
      split_f16(__ldg(q + 8) * scale, __ldg(q + 9) * scale, v.y, v.w);
    }
    wf[((int64_t)eks * NT + nt) * 32 + g * 4 + t] = v;
  }
}

// A 16-byte W fragment that skips L1: W streams through once per tile, and
// L1 keeps the producers' tables and rows (in a 16-row form of this kernel,
// 60000 rows, E = 16, 10 classes: 2.85 -> 2.82 ms against __ldg).
__device__ __forceinline__ uint4 ldg_stream_u4(const uint4* p) {
  uint4 v;
  asm("ld.global.nc.L1::no_allocate.v4.u32 {%0, %1, %2, %3}, [%4];"
      : "=r"(v.x), "=r"(v.y), "=r"(v.z), "=r"(v.w)
      : "l"(p));
  return v;
}

template <int NT>
__global__ void __launch_bounds__(kMmaThreads, kMmaBlocksPerSM) k_logits_mma(const Launch P,
                                                               const float* __restrict__ b,
                                                               float* __restrict__ logits,
                                                               int echunks) {
  constexpr int L = 10;
  using Y = Lay<L>;
  constexpr int d = Y::d;
  static_assert(Y::SLOT <= kMmaZS && kMmaZS % 32 == 8, "z row: transform slot, bank offset 8");
  static_assert(kMmaWarps * kMmaPrefetchLines >= (d / 2 + 2 * d) / 32, "prefetch covers the tables");
  static_assert(kMmaWarps * kMmaKP * 16 == d && kMmaKP % 2 == 0, "z positions per warp");
  constexpr int NS = kMmaMT * NT * 4;  // running sums per lane: (M tile, class block, entry)
  static_assert(NS <= kMmaAccS && kMmaAccS % 4 == 0, "running sums per lane");
  extern __shared__ float4 sm4[];
  float* zb = reinterpret_cast<float*>(sm4);   // [kMmaRows][kMmaZS]
  float* sums = zb + kMmaRows * kMmaZS;        // [kMmaWarps][32 lanes][kMmaAccS]
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int g = lane >> 2, t = lane & 3;
  const int C = P.C, E = P.a.E;
  const int64_t tiles = (P.a.n + kMmaRows - 1) / kMmaRows;
  const int64_t units = tiles * echunks;
  float* mysum = sums + (warp * 32 + lane) * kMmaAccS;
  bool wcls[NT];
#pragma unroll
  for (int nt = 0; nt < NT; ++nt) wcls[nt] = 8 * nt + g < C;  // the lane's class is real
  const int ks0 = kMmaKP * warp;  // cos k-steps ks0 .. ks0 + KP - 1; their sin k-steps are 64 later
  for (int64_t u = blockIdx.x; u < units; u += gridDim.x) {
    const int64_t tile = u / echunks;
    const int ch = (int)(u % echunks);
    const int e0 = E * ch / echunks, e1 = E * (ch + 1) / echunks;
#pragma unroll
    for (int i = 0; i < NS; i += 4)
      *reinterpret_cast<float4*>(mysum + i) = make_float4(0.f, 0.f, 0.f, 0.f);
    for (int e = e0; e < e1; ++e) {
      const int64_t off = (int64_t)e * d;
      {  // the next expansion's tables (permS, G, Cs: 80 lines of 128 B) into L1
        const int64_t offn = (int64_t)(e + 1 < E ? e + 1 : 0) * d;
        const int li = warp * kMmaPrefetchLines + lane;
        if (lane < kMmaPrefetchLines && li < 80) {
          const float* gsrc = P.a.GB ? P.a.GB : P.a.G;
          const char* line =
              li < 16   ? reinterpret_cast<const char*>(P.a.permS + offn / 2) + li * 128
              : li < 48 ? reinterpret_cast<const char*>(gsrc + offn) + (li - 16) * 128
                        : reinterpret_cast<const char*>(P.a.Cs + offn) + (li - 48) * 128;
          asm volatile("prefetch.global.L1 [%0];" ::"l"(line));
        }
      }
      // --------- production: z of rows warp, warp + kMmaWarps, ... ---------
      {
        // the expansion's tables, held in registers across the warp's rows
        // (Cs, needed only at the end, is read per row)
        const uint32_t bmask = __ldg(P.a.maskA + (int64_t)e * Y::T + lane);
        const uint32_t ubase = __ldg(P.a.ubase + (int64_t)e * 32 + lane);
        uint32_t poff[16];
        float gt[32];
        load_skew_offsets(P.a.permS + (int64_t)e * (d / 2), lane, poff);
        if (P.a.GB) {
          const float4* gb = reinterpret_cast<const float4*>(P.a.GB + off) + lane;
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
          for (int j = 0; j < 32; ++j) gt[j] = __ldg(P.a.G + off + Y::kB(lane, j));
        }
#pragma unroll 1
        for (int r = 0; r < kMmaRPW; ++r) {
          const int row = warp + kMmaWarps * r;
          const int64_t n = tile * kMmaRows + row;
          // a row past the batch computes the features of x = 0; its logits
          // are never written
          const bool valid = n < P.a.n;
          float* buf = zb + row * kMmaZS;
          const uint32_t slot = smem_addr(buf);
          float w[32];
          load_x_A<L>(P, n, valid, lane, w);
          apply_signs(w, bmask);
          hreg<Y::maskA()>(w);
          store_A<L>(buf, 0, lane, w);
          __syncwarp();
          load_B<L>(buf, 0, lane, w);
          hreg<Y::maskB()>(w);
          store_skew(buf, ubase, w);
          __syncwarp();
#pragma unroll
          for (int j = 0; j < 32; ++j)
            w[j] = lds32(slot + ((j & 1) ? (poff[j >> 1] >> 16) : (poff[j >> 1] & 0xffffu)));
          hreg_scaled<Y::maskB()>(w, gt);
          __syncwarp();
          store_B<L>(buf, 0, lane, w);
          __syncwarp();
          load_A<L>(buf, 0, lane, w);
          hreg<Y::maskA()>(w);
          __syncwarp();  // every lane holds its values: the slice takes z now
#pragma unroll
          for (int m = 0; m < 8; ++m) {
            const float4 c4 =
                __ldg(reinterpret_cast<const float4*>(P.a.Cs + off + Y::kA(lane, 4 * m)));
            const float2 z01 = mul2(make_float2(c4.x, c4.y), make_float2(w[4 * m], w[4 * m + 1]));
            const float2 z23 = mul2(make_float2(c4.z, c4.w), make_float2(w[4 * m + 2], w[4 * m + 3]));
            *reinterpret_cast<float4*>(buf + Y::kA(lane, 4 * m)) =
                make_float4(z01.x, z01.y, z23.x, z23.y);
          }
        }
      }
      // ------ contraction: z positions [16 KP w, 16 KP (w + 1)), KP = kMmaKP ------
      // W fragments of the first two pairs of k-steps (their L2 latency
      // overlaps the wait for the other rows); each later pair is loaded two
      // pairs ahead of its use
      const uint4* wb = P.wf + (int64_t)e * kMmaKsteps * NT * 32 + lane;
      uint4 wr[2][2][NT];  // [ring slot][cos, sin][class block]
#pragma unroll
      for (int s = 0; s < 2; ++s)
#pragma unroll
        for (int h = 0; h < 2; ++h)
#pragma unroll
          for (int nt = 0; nt < NT; ++nt)
            wr[s][h][nt] = wcls[nt] ? ldg_stream_u4(wb + ((ks0 + s + 64 * h) * NT + nt) * 32)
                                    : make_uint4(0u, 0u, 0u, 0u);
      __syncthreads();  // z of all the tile's rows is in the buffer
      float acc[NS];
#pragma unroll
      for (int i = 0; i < NS; i += 4) {
        const float4 v = *reinterpret_cast<const float4*>(mysum + i);
        acc[i] = v.x;
        acc[i + 1] = v.y;
        acc[i + 2] = v.z;
        acc[i + 3] = v.w;
      }
#pragma unroll
      for (int kk = 0; kk < kMmaKP; ++kk) {
        const int sl = kk & 1;
        uint4 wv[2][NT];
#pragma unroll
        for (int h = 0; h < 2; ++h)
#pragma unroll
          for (int nt = 0; nt < NT; ++nt) {
            wv[h][nt] = wr[sl][h][nt];
            if (kk + 2 < kMmaKP)
              wr[sl][h][nt] = wcls[nt]
                                  ? ldg_stream_u4(wb + ((ks0 + kk + 2 + 64 * h) * NT + nt) * 32)
                                  : make_uint4(0u, 0u, 0u, 0u);
          }
        const int p = 16 * (ks0 + kk) + 2 * t;  // z of the pairs (p, p + 1) and (p + 8, p + 9)
#pragma unroll
        for (int mt = 0; mt < kMmaMT; ++mt) {
          const float* z0 = zb + (16 * mt + g) * kMmaZS + p;  // row g of the M tile
          const float* z1 = z0 + 8 * kMmaZS;                   // row g + 8
          // A registers a0..a3: (row g, k 2t..), (row g + 8, k 2t..),
          // (row g, k 2t + 8..), (row g + 8, k 2t + 8..)
          float2 c[4], s[4];
          cos_sin_z2(*reinterpret_cast<const float2*>(z0), c[0], s[0]);
          cos_sin_z2(*reinterpret_cast<const float2*>(z1), c[1], s[1]);
          cos_sin_z2(*reinterpret_cast<const float2*>(z0 + 8), c[2], s[2]);
          cos_sin_z2(*reinterpret_cast<const float2*>(z1 + 8), c[3], s[3]);
          uint32_t chi[4], clo[4], shi[4], slo[4];
#pragma unroll
          for (int q = 0; q < 4; ++q) {
            split_f16(c[q].x, c[q].y, chi[q], clo[q]);
            split_f16(s[q].x, s[q].y, shi[q], slo[q]);
          }
#pragma unroll
          for (int nt = 0; nt < NT; ++nt) {
            float pr[4];
            h16::mma16816_f16_zero(pr, clo, wv[0][nt].x, wv[0][nt].y);
            h16::mma16816_f16(pr, chi, wv[0][nt].z, wv[0][nt].w);
            h16::mma16816_f16(pr, chi, wv[0][nt].x, wv[0][nt].y);
            h16::mma16816_f16(pr, slo, wv[1][nt].x, wv[1][nt].y);
            h16::mma16816_f16(pr, shi, wv[1][nt].z, wv[1][nt].w);
            h16::mma16816_f16(pr, shi, wv[1][nt].x, wv[1][nt].y);
            float* a = acc + (mt * NT + nt) * 4;
            const float2 s01 = add2(make_float2(a[0], a[1]), make_float2(pr[0], pr[1]));
            const float2 s23 = add2(make_float2(a[2], a[3]), make_float2(pr[2], pr[3]));
            a[0] = s01.x;
            a[1] = s01.y;
            a[2] = s23.x;
            a[3] = s23.y;
          }
        }
      }
#pragma unroll
      for (int i = 0; i < NS; i += 4)
        *reinterpret_cast<float4*>(mysum + i) =
            make_float4(acc[i], acc[i + 1], acc[i + 2], acc[i + 3]);
      __syncthreads();  // the buffer is free for the next expansion's rows
    }
    // ---- the warps' sums, added in a fixed order, scaled back ----
    for (int o = threadIdx.x; o < kMmaRows * C; o += kMmaThreads) {
      const int sr = o / C, cls = o % C;
      const int mt = sr >> 4, rg = sr & 7, rhi = (sr >> 3) & 1;  // M tile, row g, row g + 8
      const int nt = cls >> 3, ct = (cls & 7) >> 1, clo = cls & 1;
      const int at = (4 * rg + ct) * kMmaAccS + (mt * NT + nt) * 4 + 2 * rhi + clo;
      float v = 0.f;
#pragma unroll
      for (int qw = 0; qw < kMmaWarps; ++qw) v += sums[qw * 32 * kMmaAccS + at];
      v *= __ldg(P.winv + cls);
      const int64_t row = tile * kMmaRows + sr;
      if (row < P.a.n) {
        if (echunks == 1) logits[row * C + cls] = v + (b ? b[cls] : 0.f);
        else P.part[(row * echunks + ch) * C + cls] = v;
      }
    }
    __syncthreads();  // the sums are read before the next tile clears them
  }
}

template <int NT>
cudaError_t run_logits_mma(Launch P, const float* W, const float* b, float* scratch,
                           float* logits, cudaStream_t s) {
  const int E = P.a.E;
  uint4* wf = reinterpret_cast<uint4*>(scratch);
  float* inv = scratch + (int64_t)E * kMmaKsteps * NT * 32 * 4;
  P.wf = wf;
  P.winv = inv;
  P.part = inv + CMAX;
  k_logits_wsplit<NT><<<NT * 8, 256, 0, s>>>(W, P.C, E, wf, inv);
  cudaError_t err = cudaGetLastError();
  if (err != cudaSuccess) return err;
  const size_t smem = sizeof(float) * (kMmaRows * kMmaZS + kMmaWarps * 32 * kMmaAccS);
  err = cudaFuncSetAttribute(k_logits_mma<NT>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                             (int)smem);
  if (err != cudaSuccess) return err;
  int occ = 0;
  err = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, k_logits_mma<NT>, kMmaThreads, smem);
  if (err != cudaSuccess) return err;
  const int echunks = logits_mma_echunks(P.a.n, E, P.a.num_sms);
  const int64_t units = (P.a.n + kMmaRows - 1) / kMmaRows * echunks;
  const int64_t slots = (int64_t)P.a.num_sms * std::max(1, std::min(occ, kMmaBlocksPerSM));
  const unsigned grid = (unsigned)std::max<int64_t>(1, std::min(units, slots));
  k_logits_mma<NT><<<grid, kMmaThreads, smem, s>>>(P, b, logits, echunks);
  err = cudaGetLastError();
  if (err != cudaSuccess || echunks == 1) return err;
  const int64_t total = P.a.n * P.C;
  k_logits_reduce<<<(unsigned)((total + 255) / 256), 256, 0, s>>>(P.part, b, P.a.n, echunks, P.C,
                                                                  logits);
  return cudaGetLastError();
}

template <class K>
int occ_blocks(K kernel, int threads, size_t smem) {
  int b = 0;
  if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&b, kernel, threads, smem) != cudaSuccess)
    b = 1;
  return std::max(b, 1);
}

template <int L, int MODE>
cudaError_t run(const Launch& P, cudaStream_t s) {
  const int num_sms = P.a.num_sms;
  if constexpr (L <= 4) {
    const int occ = occ_blocks(k_feat_tiny<L, MODE>, 128, 0);
    const int64_t need = (P.a.n * P.a.E + 127) / 128;
    const unsigned grid = (unsigned)std::max<int64_t>(1, std::min<int64_t>(need, (int64_t)num_sms * occ));
    k_feat_tiny<L, MODE><<<grid, 128, 0, s>>>(P);
  } else if constexpr (L <= 10) {
    using WS = WarpShape<L>;
    const int occ = occ_blocks(k_feat_warp<L, MODE>, kWarps * 32, 0);
    const int64_t slots = (int64_t)num_sms * occ * kWarps;  // resident warps
    const int64_t full = (P.a.n + WS::SPI - 1) / WS::SPI * P.a.E;
    if constexpr (WS::R > 1) {
      // One round of VPW samples per item: chosen by the plan's launch shape,
      // else for a small batch (fewer full tiles than resident warps).
      const bool one = P.a.rows_per_item > 0 ? P.a.rows_per_item == WS::VPW : full < slots;
      if (one) {
        const int64_t items = (P.a.n + WS::VPW - 1) / WS::VPW * P.a.E;
        const unsigned grid = (unsigned)std::max<int64_t>(
            1, std::min<int64_t>((items + kWarps - 1) / kWarps, slots / kWarps));
        k_feat_warp<L, MODE, true><<<grid, kWarps * 32, 0, s>>>(P);
        return cudaGetLastError();
      }
    }
    const int64_t need = (full + kWarps - 1) / kWarps;
    const unsigned grid = (unsigned)std::max<int64_t>(1, std::min<int64_t>(need, slots / kWarps));
    k_feat_warp<L, MODE><<<grid, kWarps * 32, 0, s>>>(P);
  } else if constexpr (MODE == MODE_FEATURES && L <= 14) {
    return launch_chunked_features(P.a, P.vec_x, P.phi, s);
  } else {
    const size_t smem = sizeof(float) * Lay<L>::SLOT;
    cudaError_t err = cudaFuncSetAttribute(k_feat_cta<L, MODE>,
                                           cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (err != cudaSuccess) return err;
    const int occ = occ_blocks(k_feat_cta<L, MODE>, Lay<L>::T, smem);
    const int64_t items = P.a.n * P.a.E;
    const unsigned grid = (unsigned)std::max<int64_t>(1, std::min<int64_t>(items, (int64_t)num_sms * occ));
    k_feat_cta<L, MODE><<<grid, Lay<L>::T, smem, s>>>(P);
  }
  return cudaGetLastError();
}

template <int MODE>
cudaError_t dispatch(const Launch& P, cudaStream_t s) {
  switch (P.a.L) {
    case 1: return run<1, MODE>(P, s);
    case 2: return run<2, MODE>(P, s);
    case 3: return run<3, MODE>(P, s);
    case 4: return run<4, MODE>(P, s);
    case 5: return run<5, MODE>(P, s);
    case 6: return run<6, MODE>(P, s);
    case 7: return run<7, MODE>(P, s);
    case 8: return run<8, MODE>(P, s);
    case 9: return run<9, MODE>(P, s);
    case 10: return run<10, MODE>(P, s);
    case 11: return run<11, MODE>(P, s);
    case 12: return run<12, MODE>(P, s);
    case 13: return run<13, MODE>(P, s);
    case 14: return run<14, MODE>(P, s);
    case 15: return run<15, MODE>(P, s);
    default: return cudaErrorInvalidValue;
  }
}

Launch make_launch(const FeatureArgs& a) {
  Launch P{};
  P.a = a;
  P.vec_x = (a.in_dim % 4 == 0) && (a.ldx % 4 == 0) &&
            (reinterpret_cast<uintptr_t>(a.x) % 16 == 0);
  return P;
}

}  // namespace

cudaError_t launch_features(const FeatureArgs& a, float* phi, cudaStream_t s) {
  if (a.n == 0) return cudaSuccess;
  if (a.L > 15) return cudaErrorInvalidValue;  // multi-pass: launch_features_multipass
  Launch P = make_launch(a);
  P.phi = phi;
  return dispatch<MODE_FEATURES>(P, s);
}

int64_t logits_scratch_floats(int L, int64_t n, int E, int C, int num_sms) {
  if (L > 15) return multipass_scratch_floats(L, n, E, C, false);
  if (L != 10) return n * E * C;
  const int ec = logits_echunks(n, E, num_sms);
  return ec > 1 ? n * ec * C : 0;
}

int64_t logits_mma_scratch_floats(int64_t n, int E, int C, int num_sms) {
  const int NT = C > 8 ? 2 : 1;
  const int ec = logits_mma_echunks(n, E, num_sms);
  return (int64_t)E * kMmaKsteps * NT * 32 * 4 + CMAX + (ec > 1 ? n * ec * C : 0);
}

cudaError_t launch_logits_mma(const FeatureArgs& a, const float* W, const float* b, int C,
                              float* scratch, float* logits, cudaStream_t s) {
  if (a.n == 0) return cudaSuccess;
  if (a.L != 10 || C < 1 || C > CMAX) return cudaErrorInvalidValue;
  Launch P = make_launch(a);
  P.W = W;
  P.C = C;
  return C > 8 ? run_logits_mma<2>(P, W, b, scratch, logits, s)
               : run_logits_mma<1>(P, W, b, scratch, logits, s);
}

cudaError_t launch_logits(const FeatureArgs& a, const float* W, const float* b, int C,
                          float* part, float* logits, cudaStream_t s) {
  if (a.n == 0) return cudaSuccess;
  if (a.L > 15)  // multi-pass: `part` is the scratch for the chunk's features
    return launch_features_multipass(a, nullptr, W, b, C, logits, part, s);
  Launch P = make_launch(a);
  P.W = W;
  P.part = part;
  P.C = C;
  if (a.L == 10) {  // tile kernel: logits written directly, no partials
    if (C <= 8) {
      switch (C) {
        case 1: return run_logits_tile<1, 1>(P, b, logits, s);
        case 2: return run_logits_tile<2, 1>(P, b, logits, s);
        case 3: return run_logits_tile<3, 1>(P, b, logits, s);
        case 4: return run_logits_tile<4, 1>(P, b, logits, s);
        case 5: return run_logits_tile<5, 1>(P, b, logits, s);
        case 6: return run_logits_tile<6, 1>(P, b, logits, s);
        case 7: return run_logits_tile<7, 1>(P, b, logits, s);
        default: return run_logits_tile<8, 1>(P, b, logits, s);
      }
    }
    switch ((C + 1) / 2) {
      case 5: return run_logits_tile<5, 2>(P, b, logits, s);
      case 6: return run_logits_tile<6, 2>(P, b, logits, s);
      case 7: return run_logits_tile<7, 2>(P, b, logits, s);
      default: return run_logits_tile<8, 2>(P, b, logits, s);
    }
  }
  cudaError_t err = dispatch<MODE_LOGITS>(P, s);
  if (err != cudaSuccess) return err;
  const int64_t total = a.n * C;
  k_logits_reduce<<<(unsigned)((total + 255) / 256), 256, 0, s>>>(part, b, a.n, a.E, C, logits);
  return cudaGetLastError();
}

}  // namespace mck
