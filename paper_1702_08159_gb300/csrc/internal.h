// Private interface between the C-ABI layer (api.cu) and the kernel files.
#pragma once
#include <cuda_runtime.h>

#include <cstdint>
#include <string>

#include "../../include/mck.h"

struct mck_plan_s {
  int64_t d = 0;
  int L = 0;  // log2(d)
  int32_t E = 0;
  int32_t kernel = 0;
  double sigma = 0.0;
  int32_t matern_t = 0;
  uint64_t seed = 0;
  int device = 0;
  int num_sms = 0;
  // Device tables (natural order, see mck_plan_tables).
  uint32_t* B_bits = nullptr;  // E x words
  uint32_t* perm = nullptr;    // E x d
  float* G = nullptr;          // E x d
  float* Cs = nullptr;         // E x d
  int64_t words = 0;           // ceil(d / 32)
  // Lane-ordered copies for the warp kernels (32 <= d <= 1024), built at plan
  // time so a warp loads an expansion's tables with coalesced 128-bit loads:
  // entry (e, m, lam, q) describes element k = kB(lam, 4m+q) of layout B.
  // Lane-ordered tables (5 <= L <= 14). L <= 10: Pi as the byte offset
  // 4*pad(pi_e(k)) inside a vector slot. 11 <= L <= 14, per 1024-float chunk:
  // Pi as the word offset of pi_e(k) in the chunked block layout.
  uint32_t* permB = nullptr;   // E x d
  float* GB = nullptr;         // E x d: G_e[k]
  uint32_t* maskA = nullptr;   // E x d/32: bit j set where B_e[kA(lam, j)] = -1
  // d = 1024 only, for the forward warp kernels: u = H B x-hat is stored for
  // the Pi gather in a skewed slot (register j of lane lam at word
  // ubase[e][lam] + 33 j, so a store instruction is conflict free for any
  // per-lane bases), and the bases are chosen at plan time to spread each
  // gather instruction's 32 sources over the 32 banks.
  uint32_t* permS = nullptr;   // E x d/2: gather byte offsets into the skewed slot, two 16-bit per word
  uint32_t* ubase = nullptr;   // E x 32: word base of lane lam's registers in the skewed slot
  // d = 1024 only, the tensor-core feature kernel's tables (mma_layout.h
  // orders): B mask, G (input order) and Cs (output order) lane-ordered as
  // 8 float4 per lane, and the skewed gather tables for its u layout.
  uint32_t* mmaMask = nullptr;  // E x 32
  float* mmaG = nullptr;        // E x d
  float* mmaCs = nullptr;       // E x d
  uint32_t* mmaPerm = nullptr;  // E x d/2 packed 16-bit byte offsets
  uint32_t* mmaBase = nullptr;  // E x 32
  // Launch shape of the batched feature kernels (mck_plan_set_launch).
  int32_t rows_per_item = 0;   // 0 = automatic
  int32_t staged = -1;         // -1 = automatic
};

namespace mck {

// Thread-local error message; returns the status for convenient `return fail(...)`.
mck_status_t fail(mck_status_t s, const std::string& msg);
mck_status_t cuda_fail(cudaError_t err, const char* where);
// `p` must be device memory of `device` whose allocation holds [p, p + bytes).
mck_status_t check_device_array(const void* p, int64_t bytes, int device, const char* name);

// ---- plan.cu -------------------------------------------------------------
mck_status_t build_tables(mck_plan_s* p, cudaStream_t s);
// d = 1024: the skewed gather tables (permS, ubase) from the plan's Pi (host
// search per expansion; synchronous). No-op for other d.
mck_status_t build_skew_tables(mck_plan_s* p);
// Replace the plan's signs: B_e[k] = -1 where B[e][k] < 0 (device E x d
// floats), and rebuild the lane-ordered tables that hold them (stream-ordered).
cudaError_t set_signs(mck_plan_s* p, const float* B, cudaStream_t s);

// ---- fwht.cu -------------------------------------------------------------
// regime: one of mck_fwht_regime_t (only d = 2^16, 2^17 have a choice).
cudaError_t launch_fwht(float* x, int64_t n, int L, int num_sms, cudaStream_t s,
                        int regime = MCK_FWHT_AUTO);
// H over index bits 15..L-1 of n vectors of 2^L (FP32 column pass; 16 <= L <= 20).
cudaError_t launch_fwht_high_bits(float* x, int64_t n, int L, int num_sms, cudaStream_t s);

// ---- fwht_mma.cu -----------------------------------------------------------
bool fwht_mma_supported(int L);
cudaError_t launch_fwht_mma(float* x, int64_t n, int L, int prec, int num_sms, cudaStream_t s);

// ---- features.cu -----------------------------------------------------------
struct FeatureArgs {
  const float* x;
  int64_t n;
  int64_t in_dim;
  int64_t ldx;
  const uint32_t* B_bits;
  const uint32_t* perm;
  const float* G;
  const float* Cs;
  const uint32_t* permB;  // lane-ordered tables (warp kernels); null when absent
  const float* GB;        // null when G is overridden by the caller
  const uint32_t* maskA;
  const uint32_t* permS;  // d = 1024: skewed gather tables (see mck_plan_s); null when absent
  const uint32_t* ubase;
  const uint32_t* mmaMask;  // d = 1024: the tensor-core kernel's tables (see mck_plan_s)
  const float* mmaG;
  const float* mmaCs;
  const uint32_t* mmaPerm;
  const uint32_t* mmaBase;
  int32_t rows_per_item;  // launch shape (mck_plan_set_launch): 0 = automatic
  int32_t staged;         // -1 = automatic
  int32_t E;
  int L;
  int num_sms;
};

cudaError_t launch_features(const FeatureArgs& a, float* phi, cudaStream_t s);
// ---- features_mma.cu: d = 1024 features with the transforms on tensor cores --
// prec: MCK_BF16, MCK_FP16, MCK_BF16_SPLIT or MCK_FP16_SPLIT.
cudaError_t launch_features_mma(const FeatureArgs& a, float* phi, int prec, cudaStream_t s);
// ---- chunks.cu: features at 2^11 <= d <= 2^14 -------------------------------
cudaError_t launch_chunked_features(const FeatureArgs& a, bool vec_x, float* phi, cudaStream_t s);
// Partial logits per (sample, expansion): part is n x E x C; then logits = sum_e part + b.
// At d = 1024 the tile kernel writes logits directly and `part` is unused.
// Floats of partial logits launch_logits needs in `part` (0: none).
int64_t logits_scratch_floats(int L, int64_t n, int E, int C, int num_sms);
// Tensor-core fused logits at d = 1024 (fp16 hi/lo split contraction): the
// floats of scratch it takes (W fragments, scales, partial logits).
int64_t logits_mma_scratch_floats(int64_t n, int E, int C, int num_sms);
cudaError_t launch_logits_mma(const FeatureArgs& a, const float* W, const float* b, int C,
                              float* scratch, float* logits, cudaStream_t s);
cudaError_t launch_logits(const FeatureArgs& a, const float* W, const float* b, int C,
                          float* part, float* logits, cudaStream_t s);

// ---- large.cu: multi-pass forms (features above 2^15, the adjoint above 2^10) --
// Floats of scratch the multi-pass calls need (C > 0: fused logits).
int64_t multipass_scratch_floats(int L, int64_t n, int E, int C, bool backward);
// Features (phi) or, when logits is given, softmax-ready logits W phi + b.
cudaError_t launch_features_multipass(const FeatureArgs& a, float* phi, const float* W,
                                      const float* b, int C, float* logits, float* scratch,
                                      cudaStream_t s);
struct BackwardArgs;
cudaError_t launch_backward_multipass(const BackwardArgs& b, float* scratch, cudaStream_t s);

// ---- train.cu ------------------------------------------------------------
cudaError_t launch_softmax_xent(const float* logits, const int32_t* labels, int64_t n, int C,
                                float* loss, float* dlogits, cudaStream_t s);

struct BackwardArgs {
  FeatureArgs f;
  const float* dphi;     // n x 2Ed, or null when dlogits/W are given
  const float* W;        // C x 2Ed (fused logits backward)
  const float* dlogits;  // n x C
  int C;
  float* phi_out;  // optional n x 2Ed: recomputed features (for dW)
  float* dx;
  float* dCs;
  float* dG;
  float* dB;  // optional E x d: gradient w.r.t. the diagonal B read as real values
};
// Partial rows of dCs/dG (and dB) sums the adjoint writes: E x (blocks per expansion).
int64_t backward_partials(int L, int64_t n, int E, int num_sms);
// partials: num_partials x (dB ? 3 : 2) x d floats, num_partials = backward_partials(...).
cudaError_t launch_backward(const BackwardArgs& a, float* partials, int64_t num_partials,
                            cudaStream_t s);
cudaError_t launch_logit_weight_grads(const float* dlogits, const float* phi, int64_t n, int C,
                                      int64_t F, float* dW, float* db, cudaStream_t s);

}  // namespace mck
