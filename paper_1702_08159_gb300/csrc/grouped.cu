// Uneven batches in one persistent launch: vectors of different padded
// dimensions (32 <= d <= 2^14), kernels and expansion counts, each through
// its own plan (Sec. "McKernel": every expansion is an i.i.d. instance of
// Z-hat, so a vector may use any prefix of a plan's expansions).
//
// mck_group_create turns the items into a work list once:
//   * d <= 1024: "warp steps" -- up to 32/2^(L-5) vectors (4x as many at
//     d = 1024, 2x at 512, in rounds that share one table load) that share a
//     plan and an expansion, processed by one warp like the batched feature
//     kernel (register layouts A and B, lane-ordered tables);
//   * d >= 2048: "block items" -- one (vector, expansion) for a sub-block of
//     2^(L-5) threads in the chunked block form (one 1024-float chunk per
//     warp), each sub-block synchronising on its own named barrier.
// The work runs in phases, one per kind and size, largest items first: all
// block items of d = 2^14, then 2^13, ..., then the warp steps of d = 1024
// down to 32. Within a phase every sub-block (or warp) takes its next item
// (or `grain` steps) from the phase's own atomic counter, independently of
// the others, requesting the one after while the current runs and copying
// its record (addresses resolved at create time) into shared memory with
// cp.async; the block synchronises only between phases, where the shared
// memory is partitioned anew. The persistent kernel runs one 512-thread
// block per SM; no thread ever waits for another block. mck_group_features
// allocates nothing and never blocks the host, so it can be captured in a
// CUDA graph.
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <new>
#include <string>
#include <vector>

#include "common.cuh"
#include "internal.h"

namespace mck {
namespace {

constexpr int kGThreads = 512;
constexpr int kWarpBuf = 1152;      // floats: the largest VPW * SLOT (L = 5)
constexpr int kSmemFloats = 18432;  // max(16 warps x kWarpBuf, 512/T sub-blocks x SLOT)

// A plan's lane-ordered tables (host side, for resolving steps and items).
struct GPlan {
  const uint32_t* permB;
  const float* GB;
  const uint32_t* maskA;
  const float* Cs;
  int32_t L;
};
struct GVec {
  int64_t x_off;
  int64_t phi_off;
  int32_t in_dim;
  int32_t E;
};
// A warp step with its expansion's lane-ordered tables resolved at create time
// (pointers already offset to expansion e); its vectors' descriptors sit in
// step_vdesc[vdesc_begin ...] with phi_off already pointing at expansion e.
struct GStep {
  int64_t vdesc_begin;
  const uint32_t* permB;
  const float* GB;
  const uint32_t* maskA;
  const float* Cs;
  int32_t L;
  int32_t count;
};
struct GItem {
  int32_t vec;
  int32_t plan;
  int32_t e;
  int32_t L;
};
// A block item with its addresses resolved at create time: the expansion's
// lane-ordered tables and the vector's input and output offsets.
struct alignas(16) GItemRec {
  const uint32_t* permB;  // + e d
  const float* GB;        // + e d
  const uint32_t* maskA;  // + e d / 32
  const float* Cs;        // + e d
  int64_t x_off;
  int64_t phi_off;  // of the expansion's [cos | sin] block
  int32_t in_dim;
  int32_t pad[3];
};
static_assert(sizeof(GItemRec) == 64, "item record");
// A phase: the block items (type 1) or the warp steps (type 0) of one L.
struct GPhase {
  int64_t begin;  // into items (type 1) or steps (type 0)
  int64_t count;
  int32_t type;
  int32_t L;
};
struct GArgs {
  const GStep* steps;
  const GVec* step_vdesc;
  const GItemRec* items;
  const GPhase* phases;
  int32_t num_phases;
  int32_t grain;  // warp steps per fetch
  int* counters;  // one per phase, zero at launch
  const float* x;
  float* phi;
  bool vec_x;
};
constexpr int kMaxSubs = kGThreads >> 6;  // sub-blocks at L = 11
// Per sub-block state of a block phase, in shared memory: item indices two
// ahead (ring of 3) and the records of the current and the next item.
struct alignas(16) SubState {
  int idx[3];
  int pad;
  GItemRec rec[2];
};

__device__ __forceinline__ void apply_signs(float (&w)[32], uint32_t mask) {
#pragma unroll
  for (int j = 0; j < 32; ++j)
    w[j] = __int_as_float(__float_as_int(w[j]) ^ ((mask << (31 - j)) & 0x80000000u));
}

template <int L>
__device__ __forceinline__ void load_row_A(const float* __restrict__ row, int64_t in_dim,
                                           bool vec, bool valid, int lam, float (&w)[32]) {
#pragma unroll
  for (int m = 0; m < 8; ++m) {
    const int k0 = Lay<L>::kA(lam, 4 * m);
    float4 v = make_float4(0.f, 0.f, 0.f, 0.f);
    if (valid) {
      if (vec) {
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

template <int L>
__device__ __forceinline__ void store_features_A(float* __restrict__ out, int lam,
                                                 const float (&h)[32], const float* __restrict__ Cs) {
  constexpr int d = 1 << L;
#pragma unroll
  for (int m = 0; m < 8; ++m) {
    const int k0 = Lay<L>::kA(lam, 4 * m);
    const float4 c4 = __ldg(reinterpret_cast<const float4*>(Cs + k0));
    const float cs[4] = {c4.x, c4.y, c4.z, c4.w};
    float c[4], s[4];
    cos_sin4(cs, &h[4 * m], c, s);
    __stcs(reinterpret_cast<float4*>(out + k0), make_float4(c[0], c[1], c[2], c[3]));
    __stcs(reinterpret_cast<float4*>(out + d + k0), make_float4(s[0], s[1], s[2], s[3]));
  }
}

// Vectors per warp step: VPW = 32 / 2^(L-5) at a time, R times over (the
// tables are loaded once per step: R = 4 at d = 1024, 2 at 512, 1 below).
__host__ __device__ constexpr int step_rounds(int L) { return L >= 10 ? 4 : (L == 9 ? 2 : 1); }

// One warp step (5 <= L <= 10): group g of the warp handles vectors g,
// g + VPW, ... of the step; the tables are the step's resolved pointers (one
// dependent load less than going through the plan), the vector descriptors a
// flat array.
template <int L>
__device__ __forceinline__ void warp_step(const GArgs& a, const GStep& st, float* buf, int lane) {
  using Y = Lay<L>;
  constexpr int VPW = 32 / Y::T;
  const int g = lane / Y::T, lam = lane % Y::T;
  const uint32_t slot = smem_addr(buf) + 4u * (uint32_t)(g * Y::SLOT);
  const uint32_t bmask = __ldg(st.maskA + lam);
  uint32_t poff[16];
  float gt[32];
  const uint4* pb = reinterpret_cast<const uint4*>(st.permB) + lam;
  const float4* gb = reinterpret_cast<const float4*>(st.GB) + lam;
#pragma unroll
  for (int m = 0; m < 8; ++m) {
    const uint4 v = __ldg(pb + m * Y::T);
    poff[2 * m] = v.x | (v.y << 16);
    poff[2 * m + 1] = v.z | (v.w << 16);
    const float4 q = __ldg(gb + m * Y::T);
    gt[4 * m] = q.x;
    gt[4 * m + 1] = q.y;
    gt[4 * m + 2] = q.z;
    gt[4 * m + 3] = q.w;
  }
#pragma unroll 1
  for (int r = 0; r < step_rounds(L); ++r) {
  const int k = r * VPW + g;
  if (r * VPW >= st.count) break;
  const bool valid = k < st.count;
  GVec v{};
  if (valid) v = a.step_vdesc[st.vdesc_begin + k];
  float w[32];
  load_row_A<L>(a.x + v.x_off, v.in_dim, a.vec_x, valid, lam, w);
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
#pragma unroll
  for (int j = 0; j < 32; ++j)
    w[j] = lds32(slot + ((j & 1) ? (poff[j >> 1] >> 16) : (poff[j >> 1] & 0xffffu)));
  hreg_scaled<Y::maskB()>(w, gt);
  __syncwarp();
  if constexpr (L > 5) {
    store_B<L>(buf, g, lam, w);
    __syncwarp();
    load_A<L>(buf, g, lam, w);
  }
  hreg<Y::maskA()>(w);
  if (valid) store_features_A<L>(a.phi + v.phi_off, lam, w, st.Cs);
  __syncwarp();
  }
}

// One block item (11 <= L <= 14): the chunked block form of the map on a
// sub-block of 2^(L-5) threads (2^(L-10) warps, one 1024-float chunk each)
// that synchronises on its own named barrier `bar`.
template <int L>
__device__ __forceinline__ void block_item(const GArgs& a, const GItemRec& r, float* buf, int tid,
                                           int bar) {
  chunked_map<L>(a.x + r.x_off, r.in_dim, a.vec_x, r.permB, r.GB, nullptr, r.maskA, r.Cs,
                 a.phi + r.phi_off, buf, tid, [bar] { named_barrier(bar, Chunked<L>::NT); });
}

// A block phase: each sub-block takes items from the phase's counter until
// none are left. The index after next is requested while an item runs (the
// sub-block's first thread holds the pending result and publishes it at the
// end) and the next item's record is copied into shared memory meanwhile.
template <int L>
__device__ void block_phase(const GArgs& a, const GPhase& ph, int* ctr, float* smem,
                            SubState* subs, int tid) {
  constexpr int NT = Chunked<L>::NT;  // threads per sub-block
  const int sb = tid / NT, lam = tid % NT, bar = 1 + sb;
  SubState& S = subs[sb];
  float* buf = smem + sb * ((1 << L) + (1 << L) / 32);
  // one commit group per call and thread: item i's record into slot `slot`
  auto fetch = [&](int64_t i, int slot) {
    if (i < ph.count && lam < 4)
      cp_async16(smem_addr(reinterpret_cast<char*>(&S.rec[slot]) + 16 * lam),
                 reinterpret_cast<const char*>(a.items + ph.begin + i) + 16 * lam, 16);
    cp_async_commit();
  };
  if (lam == 0) {
    S.idx[0] = atomicAdd(ctr, 1);
    S.idx[1] = atomicAdd(ctr, 1);
  }
  named_barrier(bar, NT);
  fetch(S.idx[0], 0);
  cp_async_wait<0>();
  named_barrier(bar, NT);
  for (int k = 0;; ++k) {
    const int64_t i = S.idx[k % 3];
    if (i >= ph.count) break;
    fetch(S.idx[(k + 1) % 3], (k & 1) ^ 1);
    int next = 0;
    if (lam == 0) next = atomicAdd(ctr, 1);
    block_item<L>(a, S.rec[k & 1], buf, lam, bar);
    cp_async_wait<0>();  // the next item's record has landed
    if (lam == 0) S.idx[(k + 2) % 3] = next;
    named_barrier(bar, NT);
  }
}

// A warp phase: each warp takes `grain` steps at a time from the phase's
// counter (the next batch requested while the current one runs).
template <int L>
__device__ void warp_phase(const GArgs& a, const GPhase& ph, int* ctr, float* buf, int lane) {
  const int grain = a.grain;
  int s0 = 0;
  if (lane == 0) s0 = atomicAdd(ctr, grain);
  s0 = __shfl_sync(0xffffffffu, s0, 0);
  while (s0 < ph.count) {
    int s1 = 0;
    if (lane == 0) s1 = atomicAdd(ctr, grain);
    const int64_t end = std::min<int64_t>((int64_t)s0 + grain, ph.count);
    for (int64_t s = s0; s < end; ++s) {
      const GStep st = a.steps[ph.begin + s];
      if (s + 1 < end && lane == 0)
        asm volatile("prefetch.global.L1 [%0];" ::"l"(a.steps + ph.begin + s + 1));
      warp_step<L>(a, st, buf, lane);
    }
    s0 = __shfl_sync(0xffffffffu, s1, 0);
  }
}

__global__ void __launch_bounds__(kGThreads, 1) k_grouped(const GArgs a) {
  extern __shared__ float4 sm4[];
  float* smem = reinterpret_cast<float*>(sm4);
  __shared__ SubState s_sub[kMaxSubs];
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  for (int p = 0; p < a.num_phases; ++p) {
    const GPhase ph = a.phases[p];
    int* ctr = a.counters + p;
    if (ph.type == 1) {
      switch (ph.L) {
        case 11: block_phase<11>(a, ph, ctr, smem, s_sub, tid); break;
        case 12: block_phase<12>(a, ph, ctr, smem, s_sub, tid); break;
        case 13: block_phase<13>(a, ph, ctr, smem, s_sub, tid); break;
        case 14: block_phase<14>(a, ph, ctr, smem, s_sub, tid); break;
        default: break;
      }
    } else {
      float* buf = smem + warp * kWarpBuf;
      switch (ph.L) {
        case 5: warp_phase<5>(a, ph, ctr, buf, lane); break;
        case 6: warp_phase<6>(a, ph, ctr, buf, lane); break;
        case 7: warp_phase<7>(a, ph, ctr, buf, lane); break;
        case 8: warp_phase<8>(a, ph, ctr, buf, lane); break;
        case 9: warp_phase<9>(a, ph, ctr, buf, lane); break;
        case 10: warp_phase<10>(a, ph, ctr, buf, lane); break;
        default: break;
      }
    }
    __syncthreads();  // the next phase partitions shared memory anew
  }
}

}  // namespace
}  // namespace mck

using namespace mck;

struct mck_group_s {
  int device = 0;
  int num_sms = 1;
  int64_t x_len = 0, phi_len = 0;
  bool vec_x = true;
  int grain = 2;
  std::vector<GPlan> plans;
  std::vector<GVec> vecs;
  std::vector<GStep> steps;
  std::vector<GVec> step_vdesc;
  std::vector<GItem> items;
  std::vector<GItemRec> item_recs;
  std::vector<GPhase> phases;
  // device copies
  GStep* d_steps = nullptr;
  GVec* d_step_vdesc = nullptr;
  GItemRec* d_items = nullptr;
  GPhase* d_phases = nullptr;
  int* d_counters = nullptr;
};

namespace {

template <class T>
cudaError_t upload(T** dst, const std::vector<T>& src) {
  if (src.empty()) return cudaSuccess;
  cudaError_t err = cudaMalloc(dst, sizeof(T) * src.size());
  if (err != cudaSuccess) return err;
  return cudaMemcpy(*dst, src.data(), sizeof(T) * src.size(), cudaMemcpyHostToDevice);
}

void free_group_device(mck_group_s* g) {
  cudaFree(g->d_steps);
  cudaFree(g->d_step_vdesc);
  cudaFree(g->d_items);
  cudaFree(g->d_phases);
  cudaFree(g->d_counters);
  cudaGetLastError();
}

// The phases: block items by L (largest first), then warp steps by L (largest
// first); steps and items are sorted so that each phase is one contiguous run.
void build_phases(mck_group_s* g) {
  std::stable_sort(g->steps.begin(), g->steps.end(),
                   [](const GStep& a, const GStep& b) { return a.L > b.L; });
  std::stable_sort(g->items.begin(), g->items.end(),
                   [](const GItem& a, const GItem& b) { return a.L > b.L; });
  g->item_recs.clear();
  for (const GItem& it : g->items) {
    const GPlan& pl = g->plans[it.plan];
    const GVec& v = g->vecs[it.vec];
    const int64_t eo = (int64_t)it.e << it.L;
    g->item_recs.push_back(GItemRec{pl.permB + eo, pl.GB + eo, pl.maskA + eo / 32, pl.Cs + eo,
                                    v.x_off, v.phi_off + 2 * eo, v.in_dim, {0, 0, 0}});
  }
  g->phases.clear();
  for (int64_t b = 0; b < (int64_t)g->items.size();) {
    int64_t e = b;
    while (e < (int64_t)g->items.size() && g->items[e].L == g->items[b].L) ++e;
    g->phases.push_back(GPhase{b, e - b, 1, g->items[b].L});
    b = e;
  }
  for (int64_t b = 0; b < (int64_t)g->steps.size();) {
    int64_t e = b;
    while (e < (int64_t)g->steps.size() && g->steps[e].L == g->steps[b].L) ++e;
    g->phases.push_back(GPhase{b, e - b, 0, g->steps[b].L});
    b = e;
  }
}

mck_status_t upload_all(mck_group_s* g) {
  free_group_device(g);
  g->d_steps = nullptr;
  g->d_step_vdesc = nullptr;
  g->d_items = nullptr;
  g->d_phases = nullptr;
  g->d_counters = nullptr;
  cudaError_t err = upload(&g->d_steps, g->steps);
  if (err == cudaSuccess) err = upload(&g->d_step_vdesc, g->step_vdesc);
  if (err == cudaSuccess) err = upload(&g->d_items, g->item_recs);
  if (err == cudaSuccess) err = upload(&g->d_phases, g->phases);
  if (err == cudaSuccess && !g->phases.empty())
    err = cudaMalloc(&g->d_counters, sizeof(int) * g->phases.size());
  if (err != cudaSuccess) {
    cudaGetLastError();
    return fail(MCK_ENOMEM, "group work list upload failed");
  }
  return MCK_OK;
}

}  // namespace

extern "C" {

mck_status_t mck_group_create(mck_group_t* out, const mck_plan_t* plans, int32_t num_plans,
                              const mck_group_item_t* items, int64_t num_items, int64_t x_len,
                              int64_t phi_len, int32_t grain) {
  if (!out || !plans || (num_items > 0 && !items)) return fail(MCK_EINVAL, "NULL argument");
  if (num_plans < 1 || num_items < 0) return fail(MCK_EINVAL, "need >= 1 plan and >= 0 items");
  if (num_items > (int64_t)1 << 30) return fail(MCK_EINVAL, "too many items");
  if (grain < 0 || grain > 64) return fail(MCK_EINVAL, "grain must be in [0, 64]");
  const int device = plans[0] ? plans[0]->device : 0;
  for (int32_t p = 0; p < num_plans; ++p) {
    if (!plans[p]) return fail(MCK_EINVAL, "NULL plan");
    if (plans[p]->device != device) return fail(MCK_EINVAL, "plans on different devices");
    if (plans[p]->L < 5 || plans[p]->L > 14)
      return fail(MCK_EUNSUPPORTED, "grouped launches support 32 <= d <= 2^14");
  }
  mck_group_s* g = new (std::nothrow) mck_group_s();
  if (!g) return fail(MCK_ENOMEM, "group allocation failed");
  g->device = device;
  g->num_sms = plans[0]->num_sms;
  g->x_len = x_len;
  g->phi_len = phi_len;
  g->grain = grain ? grain : 2;
  for (int32_t p = 0; p < num_plans; ++p) {
    const mck_plan_s* q = plans[p];
    g->plans.push_back(GPlan{q->permB, q->GB, q->maskA, q->Cs, q->L});
  }
  // per-plan vector lists (for warp steps) and validation
  std::vector<std::vector<int32_t>> by_plan(num_plans);
  for (int64_t i = 0; i < num_items; ++i) {
    const mck_group_item_t& it = items[i];
    if (it.plan < 0 || it.plan >= num_plans) {
      delete g;
      return fail(MCK_EINVAL, "item " + std::to_string(i) + ": plan index out of range");
    }
    const mck_plan_s* q = plans[it.plan];
    if (it.E < 1 || it.E > q->E || it.in_dim < 1 || it.in_dim > q->d || it.x_offset < 0 ||
        it.phi_offset < 0 || it.x_offset + it.in_dim > x_len ||
        it.phi_offset + 2 * (int64_t)it.E * q->d > phi_len) {
      delete g;
      return fail(MCK_EINVAL, "item " + std::to_string(i) + ": E, in_dim or offsets out of range");
    }
    if ((it.phi_offset & 3) != 0) {
      delete g;
      return fail(MCK_EINVAL, "item " + std::to_string(i) + ": phi_offset must be a multiple of 4");
    }
    if ((it.x_offset & 3) || (it.in_dim & 3)) g->vec_x = false;
    g->vecs.push_back(GVec{it.x_offset, it.phi_offset, (int32_t)it.in_dim, it.E});
    by_plan[it.plan].push_back((int32_t)i);
  }
  for (int32_t p = 0; p < num_plans; ++p) {
    const int L = plans[p]->L;
    std::vector<int32_t>& vs = by_plan[p];
    std::stable_sort(vs.begin(), vs.end(),
                     [&](int32_t a, int32_t b) { return g->vecs[a].E > g->vecs[b].E; });
    if (L <= 10) {
      const int vpw = (32 >> (L - 5)) * step_rounds(L);  // vectors per step
      const int emax = vs.empty() ? 0 : g->vecs[vs[0]].E;
      for (int e = 0; e < emax; ++e) {
        int64_t cnt = 0;  // vectors using expansion e: a prefix of vs
        while (cnt < (int64_t)vs.size() && g->vecs[vs[cnt]].E > e) ++cnt;
        for (int64_t b = 0; b < cnt; b += vpw) {
          const int c = (int)std::min<int64_t>(vpw, cnt - b);
          const GPlan& pl = g->plans[p];
          const int64_t eo = (int64_t)e << L;
          g->steps.push_back(GStep{(int64_t)g->step_vdesc.size(), pl.permB + eo, pl.GB + eo,
                                   pl.maskA + ((int64_t)e << (L - 5)), pl.Cs + eo, L, c});
          for (int k = 0; k < c; ++k) {
            GVec v = g->vecs[vs[b + k]];
            v.phi_off += 2 * eo;  // expansion e's [cos | sin] block
            g->step_vdesc.push_back(v);
          }
        }
      }
    } else {
      for (int32_t v : vs)
        for (int e = 0; e < g->vecs[v].E; ++e) g->items.push_back(GItem{v, p, e, L});
    }
  }
  build_phases(g);
  int prev = -1;
  cudaGetDevice(&prev);
  cudaSetDevice(device);
  mck_status_t st = upload_all(g);
  if (st == MCK_OK) {
    cudaError_t err = cudaFuncSetAttribute(k_grouped, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                           (int)(sizeof(float) * kSmemFloats));
    if (err != cudaSuccess) st = cuda_fail(err, "mck_group_create");
  }
  if (prev >= 0) cudaSetDevice(prev);
  if (st != MCK_OK) {
    free_group_device(g);
    delete g;
    return st;
  }
  *out = g;
  return MCK_OK;
}

mck_status_t mck_group_set_grain(mck_group_t g, int32_t grain) {
  if (!g) return fail(MCK_EINVAL, "group is NULL");
  if (grain < 1 || grain > 64) return fail(MCK_EINVAL, "grain must be in [1, 64]");
  g->grain = grain;  // read at the next launch (a captured graph keeps its own)
  return MCK_OK;
}

mck_status_t mck_group_info(mck_group_t g, int64_t* num_units, int64_t* num_steps,
                            int64_t* num_block_items, int32_t* grain) {
  if (!g) return fail(MCK_EINVAL, "group is NULL");
  if (num_units) *num_units = (int64_t)g->phases.size();
  if (num_steps) *num_steps = (int64_t)g->steps.size();
  if (num_block_items) *num_block_items = (int64_t)g->items.size();
  if (grain) *grain = g->grain;
  return MCK_OK;
}

void mck_group_destroy(mck_group_t g) {
  if (!g) return;
  int prev = -1;
  cudaGetDevice(&prev);
  cudaSetDevice(g->device);
  cudaDeviceSynchronize();
  free_group_device(g);
  if (prev >= 0) cudaSetDevice(prev);
  delete g;
}

mck_status_t mck_group_features(mck_group_t g, const float* x, float* phi, mck_stream_t stream) {
  if (!g) return fail(MCK_EINVAL, "group is NULL");
  if (g->phases.empty()) return MCK_OK;
  if (!x || !phi) return fail(MCK_EINVAL, "x and phi must not be NULL");
  if ((uintptr_t)phi % 16) return fail(MCK_EINVAL, "phi must be 16-byte aligned");
  mck_status_t st = check_device_array(x, 4 * g->x_len, g->device, "x");
  if (st == MCK_OK) st = check_device_array(phi, 4 * g->phi_len, g->device, "phi");
  if (st != MCK_OK) return st;
  int prev = -1;
  cudaGetDevice(&prev);
  if (prev != g->device) cudaSetDevice(g->device);
  GArgs a{};
  a.steps = g->d_steps;
  a.step_vdesc = g->d_step_vdesc;
  a.items = g->d_items;
  a.phases = g->d_phases;
  a.num_phases = (int32_t)g->phases.size();
  a.grain = g->grain;
  a.counters = g->d_counters;
  a.x = x;
  a.phi = phi;
  a.vec_x = g->vec_x && ((uintptr_t)x % 16 == 0);
  cudaStream_t s = (cudaStream_t)stream;
  cudaError_t err = cudaMemsetAsync(g->d_counters, 0, sizeof(int) * g->phases.size(), s);
  if (err == cudaSuccess) {
    // every block takes part in every phase (it leaves a phase when the
    // phase's counter runs past its work)
    const int64_t work = (int64_t)g->items.size() + (int64_t)g->steps.size();
    const unsigned grid = (unsigned)std::max<int64_t>(1, std::min<int64_t>(g->num_sms, work));
    k_grouped<<<grid, kGThreads, sizeof(float) * kSmemFloats, s>>>(a);
    err = cudaGetLastError();
  }
  if (prev >= 0 && prev != g->device) cudaSetDevice(prev);
  return err == cudaSuccess ? MCK_OK : cuda_fail(err, "mck_group_features");
}

}  // extern "C"
