// Device building blocks shared by the transform, feature and adjoint kernels.
//
// A vector of d = 2^L floats (5 <= L <= 15) is held by T = 2^(L-5) threads,
// 32 registers each. Bit b of an element index k is either a "register bit"
// (selected by the register index j) or a "thread bit" (selected by the
// thread index lam within the vector's thread group). The Hadamard transform
// factorises over index bits (H_d = H_2 (x) ... (x) H_2, Sec. "Fast Walsh
// Hadamard": each level of the recursion pairs indices that differ in one
// bit), so H is applied by transforming the register bits of one layout in
// registers, moving the data through shared memory into a layout where other
// bits are register bits, and repeating until every bit was transformed once.
//
// Layout A  register bits {0,1} u [L-3, L); thread bits [2, L-3).
//           Four consecutive elements per register quad: 128-bit global
//           loads/stores, coalesced across the thread group.
// Layout B  register bits [s, s+5), s = min(2, L-5); thread bits the rest.
// Layout C  register bits [L-8, L-3) (only L >= 11).
// L <= 10: phase A transforms A's register bits outside B's, phase B all of B's.
// L >= 11: A transforms {0,1,L-3..L-1}, B [2,7), C [7, L-3).
//
// Shared memory: element k of vector slot g sits at word
//   g * SLOT + k + 4 * (k >> 7),      SLOT = d + max(4, d/32),
// i.e. four padding words after every 128. Because the thread bits and the
// register bits of an index are disjoint, each access is a per-thread base
// plus a compile-time offset, and the layout-A (128-bit) and layout-B/C
// (32-bit) accesses of a warp are free of bank conflicts for L >= 8 (2-way
// for L = 6, 7; L = 5 needs no layout moves).
#pragma once
#include <cuda_runtime.h>

#include <cstdint>

namespace mck {

constexpr float kTwoPiHi = 6.28125f;                    // 201/32, exact
constexpr float kTwoPiLo = 1.9353071795864769253e-3f;   // 2 pi - kTwoPiHi
constexpr float kInvTwoPi = 0.15915494309189533577f;

template <int L>
struct Lay {
  static_assert(L >= 5 && L <= 15, "register layouts cover 5 <= L <= 15");
  static constexpr int d = 1 << L;
  static constexpr int T = 1 << (L - 5);            // threads per vector
  static constexpr int S = (L - 5 < 2) ? (L - 5) : 2;
  static constexpr int CQ = (L >= 11) ? (L - 8) : 0;  // layout C first register bit
  static constexpr int SLOT = d + ((d / 32) > 4 ? (d / 32) : 4);  // padded words per vector

  // Element index of register j of thread lam, split into the disjoint
  // thread-selected and register-selected bits (k = k_t(lam) + k_r(j)).
  __host__ __device__ static constexpr int kA_t(int lam) { return lam << 2; }
  __host__ __device__ static constexpr int kA_r(int j) { return (j & 3) | ((j >> 2) << (L - 3)); }
  __host__ __device__ static constexpr int kB_t(int lam) {
    return (lam & ((1 << S) - 1)) | ((lam >> S) << (S + 5));
  }
  __host__ __device__ static constexpr int kB_r(int j) { return j << S; }
  __host__ __device__ static constexpr int kC_t(int lam) {
    return (lam & ((1 << CQ) - 1)) | ((lam >> CQ) << (CQ + 5));
  }
  __host__ __device__ static constexpr int kC_r(int j) { return j << CQ; }
  __host__ __device__ static constexpr int kA(int lam, int j) { return kA_t(lam) + kA_r(j); }
  __host__ __device__ static constexpr int kB(int lam, int j) { return kB_t(lam) + kB_r(j); }
  __host__ __device__ static constexpr int kC(int lam, int j) { return kC_t(lam) + kC_r(j); }
  // Index bit that register bit jb of layout A selects.
  static constexpr int a_bit(int jb) { return jb < 2 ? jb : (L - 3 + jb - 2); }
  static constexpr unsigned maskA() {
    unsigned m = 0;
    for (int jb = 0; jb < 5; ++jb) {
      const int kb = a_bit(jb);
      const bool in_b = (L <= 10) && kb >= S && kb < S + 5;
      if (!in_b) m |= 1u << jb;
    }
    return m;
  }
  static constexpr unsigned maskB() { return 31u; }
  static constexpr unsigned maskC() {
    unsigned m = 0;
    if (L >= 11)
      for (int jb = 0; jb < 5; ++jb)
        if (CQ + jb >= 7) m |= 1u << jb;
    return m;
  }
};

// Padded word offset of element k inside its vector slot (see header). For
// k = a + b with disjoint bits, pad(k) = pad(a) + pad(b).
__host__ __device__ __forceinline__ constexpr int pad(int k) { return k + 4 * (k >> 7); }

// Word offset of element k of vector slot g.
template <int L>
__host__ __device__ __forceinline__ constexpr int spos(int g, int k) {
  return g * Lay<L>::SLOT + pad(k);
}

// Packed FP32 pairs (two lanes of FP32 arithmetic per instruction). Each
// half rounds exactly like the scalar operation; a - c is formed as
// fma(c, -1, a), which is exact before its one rounding.
__device__ __forceinline__ float2 add2(float2 a, float2 c) { return __fadd2_rn(a, c); }
__device__ __forceinline__ float2 sub2(float2 a, float2 c) {
  return __ffma2_rn(c, make_float2(-1.f, -1.f), a);
}
__device__ __forceinline__ float2 mul2(float2 a, float2 c) { return __fmul2_rn(a, c); }
__device__ __forceinline__ float2 fma2(float2 a, float2 b, float2 c) { return __ffma2_rn(a, b, c); }

// One butterfly stage over register bit b >= 1: pairs (j, j+1) with bit 0
// clear are one packed operand, so two butterflies issue as one add and one
// subtract.
template <int b>
__device__ __forceinline__ void hstage2(float (&w)[32]) {
  static_assert(b >= 1 && b < 5, "packed stages need bit 0 inside the pair");
#pragma unroll
  for (int j = 0; j < 32; j += 2) {
    if (!(j >> b & 1)) {
      const int jc = j | (1 << b);
      const float2 a = make_float2(w[j], w[j + 1]), c = make_float2(w[jc], w[jc + 1]);
      const float2 s = add2(a, c), t = sub2(a, c);
      w[j] = s.x;
      w[j + 1] = s.y;
      w[jc] = t.x;
      w[jc + 1] = t.y;
    }
  }
}

// H over the register bits in MASK (unnormalised butterflies), bit 0 first
// (scalar: its pairs share one packed operand), then bits 1..4 packed.
template <unsigned MASK>
__device__ __forceinline__ void hreg(float (&w)[32]) {
  if constexpr ((MASK & 1u) != 0) {
#pragma unroll
    for (int j = 0; j < 32; j += 2) {
      const float a = w[j], c = w[j + 1];
      w[j] = a + c;
      w[j + 1] = a - c;
    }
  }
  if constexpr ((MASK & 2u) != 0) hstage2<1>(w);
  if constexpr ((MASK & 4u) != 0) hstage2<2>(w);
  if constexpr ((MASK & 8u) != 0) hstage2<3>(w);
  if constexpr ((MASK & 16u) != 0) hstage2<4>(w);
}

template <unsigned MASK>
__host__ __device__ constexpr int lowest_bit() {
  return (MASK & 1u) ? 0 : (MASK & 2u) ? 1 : (MASK & 4u) ? 2 : (MASK & 8u) ? 3 : 4;
}

// H over MASK applied to (s * w): the scale is folded into the first
// butterfly stage (a' = s_a w_a + s_c w_c, c' = s_a w_a - s_c w_c).
template <unsigned MASK>
__device__ __forceinline__ void hreg_scaled(float (&w)[32], const float (&s)[32]) {
  static_assert(MASK != 0, "scaled transform needs at least one bit");
  constexpr int b0 = lowest_bit<MASK>();
  if constexpr (b0 == 0) {
#pragma unroll
    for (int j = 0; j < 32; j += 2) {
      const float a = s[j] * w[j];
      const float c = w[j + 1];
      w[j] = fmaf(s[j + 1], c, a);
      w[j + 1] = fmaf(-s[j + 1], c, a);
    }
  } else {
    // packed: a = s_a w_a as one product, then c' = a -/+ s_c w_c as fmas
#pragma unroll
    for (int j = 0; j < 32; j += 2) {
      if (!(j >> b0 & 1)) {
        const int jc = j | (1 << b0);
        const float2 a = mul2(make_float2(s[j], s[j + 1]), make_float2(w[j], w[j + 1]));
        const float2 sc = make_float2(s[jc], s[jc + 1]), c = make_float2(w[jc], w[jc + 1]);
        const float2 p = fma2(sc, c, a);
        const float2 m = fma2(make_float2(-sc.x, -sc.y), c, a);
        w[j] = p.x;
        w[j + 1] = p.y;
        w[jc] = m.x;
        w[jc + 1] = m.y;
      }
    }
  }
  hreg<MASK & ~(1u << b0)>(w);
}

// cos and sin of z: z is reduced to r = z - 2 pi k in [-pi, pi] (Cody & Waite
// two-constant reduction, both products exact for |k| < 2^15), then the
// hardware approximations, whose absolute error is below 2^-21 on [-pi, pi].
__device__ __forceinline__ void cos_sin(float z, float& c, float& s) {
  const float k = rintf(z * kInvTwoPi);
  float r = fmaf(-k, kTwoPiHi, z);
  r = fmaf(-k, kTwoPiLo, r);
  c = __cosf(r);
  s = __sinf(r);
}

// cos and sin of two values z at once: the arithmetic of cos_sin (with -k =
// rint(-z / 2 pi), exact since rounding to nearest is symmetric), the
// reductions as packed pairs.
__device__ __forceinline__ void cos_sin_z2(float2 z, float2& c, float2& s) {
  const float2 t = mul2(z, make_float2(-kInvTwoPi, -kInvTwoPi));
  const float2 kn = make_float2(rintf(t.x), rintf(t.y));
  float2 r = fma2(kn, make_float2(kTwoPiHi, kTwoPiHi), z);
  r = fma2(kn, make_float2(kTwoPiLo, kTwoPiLo), r);
  c = make_float2(__cosf(r.x), __cosf(r.y));
  s = make_float2(__sinf(r.x), __sinf(r.y));
}

// cos and sin of z = cs * h for two values at once (z rounded to float32).
__device__ __forceinline__ void cos_sin2(float2 cs, float2 h, float2& c, float2& s) {
  cos_sin_z2(mul2(cs, h), c, s);
}

// cos and sin of cs[q] * h[q] for a register quad.
__device__ __forceinline__ void cos_sin4(const float* cs, const float* h, float (&c)[4],
                                         float (&s)[4]) {
  float2 c0, s0, c1, s1;
  cos_sin2(make_float2(cs[0], cs[1]), make_float2(h[0], h[1]), c0, s0);
  cos_sin2(make_float2(cs[2], cs[3]), make_float2(h[2], h[3]), c1, s1);
  c[0] = c0.x; c[1] = c0.y; c[2] = c1.x; c[3] = c1.y;
  s[0] = s0.x; s[1] = s0.y; s[2] = s1.x; s[3] = s1.y;
}

__device__ __forceinline__ uint32_t smem_addr(const void* p) {
  return static_cast<uint32_t>(__cvta_generic_to_shared(p));
}

// 16-byte asynchronous copy from global to shared memory, cached in L2 only.
// With bytes < 16 the rest of the destination is zero-filled (bytes = 0
// reads nothing). Completion is tracked per thread by commit groups.
__device__ __forceinline__ void cp_async16(uint32_t dst, const void* src, int bytes) {
  asm volatile("cp.async.cg.shared.global [%0], [%1], 16, %2;\n" ::"r"(dst), "l"(src), "r"(bytes)
               : "memory");
}
// Ask L2 for `bytes` (a multiple of 16) from global address p (16-byte
// aligned) without waiting: a hint, no registers or shared memory held.
__device__ __forceinline__ void prefetch_l2_bulk(const void* p, uint32_t bytes) {
  asm volatile("cp.async.bulk.prefetch.L2.global [%0], %1;" ::"l"(p), "r"(bytes) : "memory");
}
__device__ __forceinline__ void cp_async_commit() {
  asm volatile("cp.async.commit_group;\n" ::: "memory");
}
// Wait until at most N of this thread's most recent commit groups are pending.
template <int N>
__device__ __forceinline__ void cp_async_wait() {
  asm volatile("cp.async.wait_group %0;\n" ::"n"(N) : "memory");
}

__device__ __forceinline__ void sts32(uint32_t addr, float v) {
  asm volatile("st.shared.f32 [%0], %1;" ::"r"(addr), "f"(v) : "memory");
}
__device__ __forceinline__ float lds32(uint32_t addr) {
  float v;
  asm volatile("ld.shared.f32 %0, [%1];" : "=f"(v) : "r"(addr) : "memory");
  return v;
}
// Named barriers (ids 1..15; id 0 is __syncthreads). `threads` counts every
// thread that takes part, arriving or waiting, in whole warps. bar.sync waits;
// bar.arrive only signals, and the memory accesses before it are visible to
// the threads that waited on the same barrier.
__device__ __forceinline__ void named_barrier(int id, int threads) {
  asm volatile("bar.sync %0, %1;" ::"r"(id), "r"(threads) : "memory");
}
__device__ __forceinline__ void named_arrive(int id, int threads) {
  asm volatile("bar.arrive %0, %1;" ::"r"(id), "r"(threads) : "memory");
}
// ---------------------------------------------------------------------------
// Layout moves through shared memory. `buf` points at the caller's shared
// buffer; g is the vector slot of this thread's group. Callers separate a
// store phase from the next load phase with the appropriate barrier.
// ---------------------------------------------------------------------------
template <int L>
__device__ __forceinline__ void store_A(float* buf, int g, int lam, const float (&w)[32]) {
  float* p = buf + g * Lay<L>::SLOT + pad(Lay<L>::kA_t(lam));
#pragma unroll
  for (int m = 0; m < 8; ++m)
    *reinterpret_cast<float4*>(p + pad(Lay<L>::kA_r(4 * m))) =
        make_float4(w[4 * m], w[4 * m + 1], w[4 * m + 2], w[4 * m + 3]);
}
template <int L>
__device__ __forceinline__ void load_A(const float* buf, int g, int lam, float (&w)[32]) {
  const float* p = buf + g * Lay<L>::SLOT + pad(Lay<L>::kA_t(lam));
#pragma unroll
  for (int m = 0; m < 8; ++m) {
    const float4 v = *reinterpret_cast<const float4*>(p + pad(Lay<L>::kA_r(4 * m)));
    w[4 * m] = v.x;
    w[4 * m + 1] = v.y;
    w[4 * m + 2] = v.z;
    w[4 * m + 3] = v.w;
  }
}
template <int L>
__device__ __forceinline__ void store_B(float* buf, int g, int lam, const float (&w)[32]) {
  float* p = buf + g * Lay<L>::SLOT + pad(Lay<L>::kB_t(lam));
#pragma unroll
  for (int j = 0; j < 32; ++j) p[pad(Lay<L>::kB_r(j))] = w[j];
}
template <int L>
__device__ __forceinline__ void load_B(const float* buf, int g, int lam, float (&w)[32]) {
  const float* p = buf + g * Lay<L>::SLOT + pad(Lay<L>::kB_t(lam));
#pragma unroll
  for (int j = 0; j < 32; ++j) w[j] = p[pad(Lay<L>::kB_r(j))];
}
template <int L>
__device__ __forceinline__ void store_C(float* buf, int lam, const float (&w)[32]) {
  float* p = buf + pad(Lay<L>::kC_t(lam));
#pragma unroll
  for (int j = 0; j < 32; ++j) p[pad(Lay<L>::kC_r(j))] = w[j];
}
template <int L>
__device__ __forceinline__ void load_C(const float* buf, int lam, float (&w)[32]) {
  const float* p = buf + pad(Lay<L>::kC_t(lam));
#pragma unroll
  for (int j = 0; j < 32; ++j) w[j] = p[pad(Lay<L>::kC_r(j))];
}

// ---------------------------------------------------------------------------
// Chunked block form of the feature map for 11 <= L <= 14: a (sub-)block of
// W = 2^(L-10) warps owns one vector-expansion; warp w owns the 1024-float
// chunk w (elements 1024 w .. 1024 w + 1023) and transforms its index bits
// 0..9 exactly like the d = 1024 warp kernel (layouts A and B, warp-local
// moves through its 1056-word slot); index bits 10..L-1 are transformed
// across the chunks by threads that own columns c of all W slots. The Pi
// gather reads the whole vector from the slots through word offsets made at
// plan time. Four block barriers per vector-expansion.
// ---------------------------------------------------------------------------
template <int L>
struct Chunked {
  static_assert(L >= 11 && L <= 14, "chunked block form");
  static constexpr int W = 1 << (L - 10);                  // warps (chunks)
  static constexpr int NT = 32 * W;                        // threads
  static constexpr int VEC = (1024 / NT) >= 4 ? 4 : 2;     // columns per vector access
  static constexpr int CG = 1024 / (NT * VEC);             // column groups per thread
  static constexpr int SLOT = Lay<10>::SLOT;               // words per chunk slot
  static constexpr int WORDS = W * SLOT;
};

template <int VEC>
__device__ __forceinline__ void ld_vec(const float* p, float (&v)[VEC]) {
  if constexpr (VEC == 4) {
    const float4 t = *reinterpret_cast<const float4*>(p);
    v[0] = t.x; v[1] = t.y; v[2] = t.z; v[3] = t.w;
  } else {
    const float2 t = *reinterpret_cast<const float2*>(p);
    v[0] = t.x; v[1] = t.y;
  }
}
template <int VEC>
__device__ __forceinline__ void st_vec(float* p, const float (&v)[VEC]) {
  if constexpr (VEC == 4) *reinterpret_cast<float4*>(p) = make_float4(v[0], v[1], v[2], v[3]);
  else *reinterpret_cast<float2*>(p) = make_float2(v[0], v[1]);
}

// H over index bits 10..L-1 of the vector held in the W slots, in place
// (thread tid owns column groups tid, tid + NT, ...).
template <int L>
__device__ __forceinline__ void chunk_columns_inplace(float* sm, int tid) {
  using C = Chunked<L>;
#pragma unroll
  for (int q = 0; q < C::CG; ++q) {
    const int c0 = C::VEC * (tid + C::NT * q);
    float u[C::W][C::VEC];
#pragma unroll
    for (int i = 0; i < C::W; ++i) ld_vec<C::VEC>(sm + i * C::SLOT + pad(c0), u[i]);
#pragma unroll
    for (int h = 1; h < C::W; h <<= 1)
#pragma unroll
      for (int i = 0; i < C::W; ++i)
        if (!(i & h))
#pragma unroll
          for (int v = 0; v < C::VEC; v += 2) {
            const float2 a = make_float2(u[i][v], u[i][v + 1]);
            const float2 b = make_float2(u[i | h][v], u[i | h][v + 1]);
            const float2 s = add2(a, b), t = sub2(a, b);
            u[i][v] = s.x; u[i][v + 1] = s.y;
            u[i | h][v] = t.x; u[i | h][v + 1] = t.y;
          }
#pragma unroll
    for (int i = 0; i < C::W; ++i) st_vec<C::VEC>(sm + i * C::SLOT + pad(c0), u[i]);
  }
}

// The tables a warp of the chunked block form holds for its chunk of one
// expansion: the B mask of its lanes, the Pi word offsets (packed two per
// register) and G (lane-ordered, or natural order when overridden).
struct ChunkTabs {
  uint32_t bmask;
  uint32_t poff[16];
  float gt[32];
};

template <int L>
__device__ __forceinline__ void load_chunk_tabs(const uint32_t* __restrict__ permB,
                                                const float* __restrict__ GB,
                                                const float* __restrict__ Gnat,
                                                const uint32_t* __restrict__ maskA, int tid,
                                                ChunkTabs& t) {
  using Y = Lay<10>;
  const int warp = tid >> 5, lane = tid & 31;
  const int co = warp * 1024;
  t.bmask = __ldg(maskA + warp * 32 + lane);
  const uint4* pb = reinterpret_cast<const uint4*>(permB + co) + lane;
#pragma unroll
  for (int m = 0; m < 8; ++m) {
    const uint4 v = __ldg(pb + m * 32);
    t.poff[2 * m] = v.x | (v.y << 16);
    t.poff[2 * m + 1] = v.z | (v.w << 16);
  }
  if (Gnat) {
#pragma unroll
    for (int j = 0; j < 32; ++j) t.gt[j] = __ldg(Gnat + co + Y::kB(lane, j));
  } else {
    const float4* gb = reinterpret_cast<const float4*>(GB + co) + lane;
#pragma unroll
    for (int m = 0; m < 8; ++m) {
      const float4 v = __ldg(gb + m * 32);
      t.gt[4 * m] = v.x;
      t.gt[4 * m + 1] = v.y;
      t.gt[4 * m + 2] = v.z;
      t.gt[4 * m + 3] = v.w;
    }
  }
}

// The whole feature map of one vector-expansion in the chunked block form,
// with the expansion's tables already in registers (`t`, see
// load_chunk_tabs); Cs natural order (offset by e d). `out` receives
// [cos z | sin z] (2d floats). `bar` synchronises the NT threads of the
// (sub-)block.
// STAGED: the caller has copied x-hat into shared memory with cp.async (xs:
// this warp's 1024-float chunk, zero past in_dim, in one commit group that
// it has waited for) and Cs (css: the expansion's d values, in a commit
// group no later than the one before `next`'s). The warp reads its chunk,
// then calls `next` (which queues the next row's copies into xs); the
// output stage waits for all but the newest commit group.
template <int L, bool STAGED, class Bar, class Next>
__device__ __forceinline__ void chunked_body(const ChunkTabs& t, const float* __restrict__ xrow,
                                             int64_t in_dim, bool vec_x,
                                             const float* __restrict__ cs,
                                             float* __restrict__ out, float* sm, int tid, Bar bar,
                                             const float* xs, const float* css, Next next) {
  using C = Chunked<L>;
  using Y = Lay<10>;
  constexpr int d = 1 << L;
  const int warp = tid >> 5, lane = tid & 31;
  float* slot = sm + warp * C::SLOT;
  const uint32_t sbase = smem_addr(sm);
  const int co = warp * 1024;
  const uint32_t bmask = t.bmask;
  // u = H B x-hat: index bits 0..9 per warp, then 10..L-1 across the chunks
  {
    float w[32];
    if constexpr (STAGED) {
      __syncwarp();  // every lane has waited for its own copies of the chunk
#pragma unroll
      for (int m = 0; m < 8; ++m) {
        const float4 v = *reinterpret_cast<const float4*>(xs + Y::kA(lane, 4 * m));
        w[4 * m] = v.x;
        w[4 * m + 1] = v.y;
        w[4 * m + 2] = v.z;
        w[4 * m + 3] = v.w;
      }
      __syncwarp();  // the chunk is read before the next item's copies land
      next();
    } else {
#pragma unroll
      for (int m = 0; m < 8; ++m) {
        const int k0 = co + Y::kA(lane, 4 * m);
        float4 v = make_float4(0.f, 0.f, 0.f, 0.f);
        if (vec_x) {
          if (k0 < in_dim) v = __ldg(reinterpret_cast<const float4*>(xrow + k0));
        } else {
          if (k0 + 0 < in_dim) v.x = __ldg(xrow + k0 + 0);
          if (k0 + 1 < in_dim) v.y = __ldg(xrow + k0 + 1);
          if (k0 + 2 < in_dim) v.z = __ldg(xrow + k0 + 2);
          if (k0 + 3 < in_dim) v.w = __ldg(xrow + k0 + 3);
        }
        w[4 * m] = v.x;
        w[4 * m + 1] = v.y;
        w[4 * m + 2] = v.z;
        w[4 * m + 3] = v.w;
      }
    }
#pragma unroll
    for (int j = 0; j < 32; ++j)
      w[j] = __int_as_float(__float_as_int(w[j]) ^ ((bmask << (31 - j)) & 0x80000000u));
    hreg<Y::maskA()>(w);
    store_A<10>(slot, 0, lane, w);
    __syncwarp();
    load_B<10>(slot, 0, lane, w);
    hreg<Y::maskB()>(w);
    __syncwarp();
    store_B<10>(slot, 0, lane, w);
  }
  bar();
  chunk_columns_inplace<L>(sm, tid);
  bar();
  // v = Pi u gathered into chunk `warp` (layout B), G, H over bits 0..9
  float w[32];
#pragma unroll
  for (int j = 0; j < 32; ++j)
    w[j] = lds32(sbase + 4u * ((j & 1) ? (t.poff[j >> 1] >> 16) : (t.poff[j >> 1] & 0xffffu)));
  hreg_scaled<Y::maskB()>(w, t.gt);
  bar();  // every warp has gathered: the slots may be rewritten
  store_B<10>(slot, 0, lane, w);
  __syncwarp();
  load_A<10>(slot, 0, lane, w);
  hreg<Y::maskA()>(w);
  __syncwarp();
  store_A<10>(slot, 0, lane, w);
  if constexpr (STAGED) cp_async_wait<1>();  // this thread's Cs copies have landed (older group)
  bar();
  // bits 10..L-1 of the second transform, then z = Cs h and [cos | sin]
#pragma unroll
  for (int q = 0; q < C::CG; ++q) {
    const int c0 = C::VEC * (tid + C::NT * q);
    float u[C::W][C::VEC];
#pragma unroll
    for (int i = 0; i < C::W; ++i) ld_vec<C::VEC>(sm + i * C::SLOT + pad(c0), u[i]);
#pragma unroll
    for (int h = 1; h < C::W; h <<= 1)
#pragma unroll
      for (int i = 0; i < C::W; ++i)
        if (!(i & h))
#pragma unroll
          for (int v = 0; v < C::VEC; v += 2) {
            const float2 a = make_float2(u[i][v], u[i][v + 1]);
            const float2 b = make_float2(u[i | h][v], u[i | h][v + 1]);
            const float2 s = add2(a, b), t = sub2(a, b);
            u[i][v] = s.x; u[i][v + 1] = s.y;
            u[i | h][v] = t.x; u[i | h][v + 1] = t.y;
          }
#pragma unroll
    for (int i = 0; i < C::W; ++i) {
      const int k = c0 + 1024 * i;
      float cv[C::VEC], cz[C::VEC], sz[C::VEC];
      if constexpr (STAGED) ld_vec<C::VEC>(css + k, cv);
      else ld_vec<C::VEC>(cs + k, cv);
#pragma unroll
      for (int v = 0; v < C::VEC; v += 2) {
        float2 c2, s2;
        cos_sin2(make_float2(cv[v], cv[v + 1]), make_float2(u[i][v], u[i][v + 1]), c2, s2);
        cz[v] = c2.x; cz[v + 1] = c2.y;
        sz[v] = s2.x; sz[v + 1] = s2.y;
      }
      if constexpr (C::VEC == 4) {
        __stcs(reinterpret_cast<float4*>(out + k), make_float4(cz[0], cz[1], cz[2], cz[3]));
        __stcs(reinterpret_cast<float4*>(out + d + k), make_float4(sz[0], sz[1], sz[2], sz[3]));
      } else {
        __stcs(reinterpret_cast<float2*>(out + k), make_float2(cz[0], cz[1]));
        __stcs(reinterpret_cast<float2*>(out + d + k), make_float2(sz[0], sz[1]));
      }
    }
  }
  bar();  // the slots (and Cs) are read before the next item rewrites them
}

// Tables and map together (one vector-expansion).
template <int L, class Bar>
__device__ __forceinline__ void chunked_map(const float* __restrict__ xrow, int64_t in_dim,
                                            bool vec_x, const uint32_t* __restrict__ permB,
                                            const float* __restrict__ GB,
                                            const float* __restrict__ Gnat,
                                            const uint32_t* __restrict__ maskA,
                                            const float* __restrict__ cs, float* __restrict__ out,
                                            float* sm, int tid, Bar bar) {
  ChunkTabs t;
  load_chunk_tabs<L>(permB, GB, Gnat, maskA, tid, t);
  chunked_body<L, false>(t, xrow, in_dim, vec_x, cs, out, sm, tid, bar, nullptr, nullptr, [] {});
}

}  // namespace mck
