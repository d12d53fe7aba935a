/*
 * mck.h -- C ABI of the GB300 McKernel / Fastfood feature-map library (libmck.so).
 *
 * The library computes the random-feature map of McKernel (arXiv 1702.08159):
 *
 *   Z-hat = (1/(sigma sqrt d)) C H G Pi H B                      (Eq. etn:mckernel)
 *   phi(x) = [cos(Z-hat x-hat), sin(Z-hat x-hat)] per expansion  (Eq. etn:mcfeatures)
 *
 * with x-hat = x zero-padded to d = 2^L (Fig. 1 caption), E independent
 * expansions (Sec. "McKernel": Z-hat is instantiated E times), and
 * the classifier softmax(W phi + b) of Sec. "Empirical Analysis and
 * Experiments". B (signs), Pi (permutation), G (Gaussian) and the calibration
 * C are recreated from a seed by a counter-based hash (Sec. "API
 * Description": parameters are deterministic functions of a hash, nothing is
 * stored).
 *
 * Conventions shared by every entry point
 * ---------------------------------------
 * - All array arguments are DEVICE pointers (CUDA global memory on the plan's
 *   device), owned by the caller; the library never frees or retains them.
 *   The only exception is mck_plan_tables, which fills HOST buffers.
 * - Arrays are dense row-major float32 (int32 for labels). The feature row
 *   of one sample holds E blocks of [cos (d values) | sin (d values)], so a
 *   feature matrix is n x (2 E d) with leading dimension 2 E d.
 * - x is n x in_dim with leading dimension ldx >= in_dim (elements).
 * - Cs is the calibration already scaled by 1/(sigma sqrt d): Cs = C/(sigma sqrt d),
 *   E x d. G is E x d. Passing NULL for Cs or G uses the plan's own tables;
 *   passing arrays lets training code learn them (Sec. "Empirical Analysis":
 *   learning C and G by backpropagation).
 * - `stream` is a cudaStream_t (NULL = the legacy default stream). Every
 *   compute call is asynchronous on that stream; the library may allocate
 *   stream-ordered scratch memory on it (cudaMallocFromPoolAsync from a
 *   memory pool the library makes per device on first use, which keeps up
 *   to 1 GiB mapped between calls so that a call after a synchronisation
 *   does not map its scratch anew; the default pool is left untouched).
 *   After a context reset (cudaDeviceReset) every later call is invalid, as
 *   plans are.
 * - Gradients are written (not accumulated). Reductions over the batch (dCs,
 *   dG, dW, db) are deterministic: the same inputs give bit-identical outputs.
 * - Every call returns an mck_status_t. On failure mck_last_error() gives a
 *   message for the calling thread. Argument errors are detected before any
 *   device work is queued. MCK_ECUDA reports a CUDA runtime error.
 * - Sizes: 2 <= d <= 2^20 for plans (Matern: d <= 2^15); n >= 0 (n = 0 is a
 *   no-op). Above d = 2^15 the features run in passes over HBM scratch
 *   (stream-ordered, at most 256 MiB); see mck_features.
 */
#ifndef MCK_H
#define MCK_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct mck_plan_s* mck_plan_t; /* opaque; owns the device tables of one parameter set */
typedef void* mck_stream_t;            /* a cudaStream_t */

typedef enum {
  MCK_RBF = 0,    /* Gaussian RBF kernel exp(-|x-x'|^2/(2 sigma^2)) (Eq. etn:rbf) */
  MCK_MATERN = 1, /* RBF Matern: C_kk = |sum of t uniform unit-ball points| (Sec. "Customizing McKernel") */
  MCK_LAPLACE = 2 /* Laplacian exp(-|x-x'|/sigma): C_kk ~ chi_d/|N(0,1)|, the spherical Cauchy radius,
                     one more radial spectral distribution (Sec. "McKernel", item C) */
} mck_kernel_t;

typedef enum {
  MCK_OK = 0,
  MCK_EINVAL = -1,       /* an argument is out of range, NULL or misaligned */
  MCK_ENOMEM = -2,       /* a device or host allocation failed */
  MCK_ECUDA = -3,        /* the CUDA runtime reported an error */
  MCK_ETIMEOUT = -4,     /* a bounded device wait gave up */
  MCK_EUNSUPPORTED = -5  /* valid request this version does not implement */
} mck_status_t;

typedef enum {
  MCK_FP32 = 0,       /* float32 butterflies */
  MCK_BF16 = 1,       /* H16 digits as bf16 tensor-core products, FP32 accumulation */
  MCK_FP16 = 2,       /* the same with fp16 operands */
  MCK_BF16_SPLIT = 3, /* bf16 with each operand split into hi + lo halves (two products) */
  MCK_FP16_SPLIT = 4  /* fp16 with the hi + lo split */
} mck_prec_t;

#define MCK_MAX_LOG2_D 20          /* largest plan dimension: d = 2^20 */
#define MCK_MAX_LOG2_D_MATERN 15   /* largest Matern plan: d = 2^15 (t d^2 draws per expansion) */
#define MCK_MAX_LOG2_D_FWHT 20     /* largest standalone transform: d = 2^20 */
#define MCK_MAX_CLASSES 16         /* largest class count of the fused logit kernels */

/* Create a plan: the tables B, Pi, G and C of E expansions of dimension d,
 * recreated from `seed` (Sec. "McKernel" items B, Pi, G, C; Sec. "API
 * Description": factory pattern, parameters from a hash).
 *   d       padded dimension, a power of two, 2 <= d <= 2^20 (Matern: <= 2^15)
 *   E       number of expansions, 1 <= E <= 65536
 *   kernel  MCK_RBF, MCK_MATERN or MCK_LAPLACE
 *   sigma   kernel width, finite and > 0 (the sigma of Eq. etn:mckernel)
 *   seed    64-bit hash key; equal seeds give bit-identical B and Pi
 * The Matern order t defaults to 40 (the paper's experiments, Fig. 2-4
 * captions). The plan is created on the current CUDA device. The call is
 * synchronous: the tables are ready when it returns. *out is set only on
 * success. Errors: MCK_EINVAL (bad argument, NULL out), MCK_EUNSUPPORTED
 * (d > 2^20, or a Matern plan above 2^15), MCK_ENOMEM, MCK_ECUDA. For
 * d > 2^15 the permutations are drawn on the host (the same draws and swaps). */
mck_status_t mck_plan(mck_plan_t* out, int64_t d, int32_t E, int32_t kernel, double sigma,
                      uint64_t seed);

/* As mck_plan, with the Matern order t (1 <= t <= 4096; ignored for RBF and Laplace) and
 * the CUDA device index (-1 = current device). */
mck_status_t mck_plan_ex(mck_plan_t* out, int64_t d, int32_t E, int32_t kernel, double sigma,
                         int32_t matern_t, uint64_t seed, int32_t device);

/* Release a plan and its device tables (synchronises the device first so no
 * queued call still reads them). NULL is ignored. */
void mck_plan_destroy(mck_plan_t plan);

/* Report the parameters of a plan; any output pointer may be NULL. */
mck_status_t mck_plan_info(mck_plan_t plan, int64_t* d, int32_t* E, int32_t* kernel,
                           double* sigma, int32_t* matern_t, uint64_t* seed, int32_t* device);

/* Copy the plan's tables to HOST buffers (any may be NULL); synchronous.
 *   B_bits  E x ceil(d/32) uint32: bit (k mod 32) of word k/32 is 1 where B_e[k] = -1
 *   perm    E x d uint32: pi_e(k), with (Pi v)_k = v_{pi(k)} (Sec. "McKernel", Pi)
 *   G       E x d float32 (Sec. "McKernel", G)
 *   Cs      E x d float32: C/(sigma sqrt d) (Eq. etn:mckernel) */
mck_status_t mck_plan_tables(mck_plan_t plan, uint32_t* B_bits, uint32_t* perm, float* G,
                             float* Cs);

/* Launch shape of the batched feature kernels (mck_features, and
 * mck_fused_logits at d != 1024) for this plan: a tunable. Every shape gives
 * bit-identical results; paper_1702_08159_gb300/tune.py picks the fastest per
 * workload.
 *   rows_per_item  samples one work item covers with one load of an
 *                  expansion's tables. 0 = automatic. 32 <= d <= 1024:
 *                  32 / (d / 32) (one round of the warp's vectors, at least 1)
 *                  or max(4, that) (a full tile). 2^11 <= d <= 2^14: 1, 2 or 4.
 *   staged         -1 = automatic, 0 = off, 1 = on: the block copies the next
 *                  row's input and the expansion's Cs into shared memory with
 *                  cp.async ahead of use (2^11 <= d <= 2^14; rows that are not
 *                  16-byte aligned with in_dim % 4 == 0 run unstaged).
 * Other values, or anything but (0, -1) at other d, return MCK_EINVAL. Host
 * only: calls queued afterwards use the new shape; do not change it while
 * another thread launches work with the plan. */
mck_status_t mck_plan_set_launch(mck_plan_t plan, int32_t rows_per_item, int32_t staged);

/* The plan's launch shape (as set; 0 / -1 = automatic); outputs may be NULL. */
mck_status_t mck_plan_get_launch(mck_plan_t plan, int32_t* rows_per_item, int32_t* staged);

/* Replace the plan's sign diagonals B (Sec. "Empirical Analysis": learning
 * B, which the paper likens to attention; a trainer keeps real values and
 * uses their signs).
 *   B  device E x d float32: B_e[k] becomes -1 where B[e][k] < 0 and +1
 *      otherwise (0 and NaN give +1).
 * Stream-ordered on `stream`: work queued after it on that stream sees the
 * new signs; the caller orders other streams, and must not change the signs
 * while a group or a captured graph that uses the plan runs. Returns
 * MCK_EINVAL for a NULL plan or B. Pi, G and C are unchanged. */
mck_status_t mck_plan_set_signs(mck_plan_t plan, const float* B, mck_stream_t stream);

/* In-place unnormalised Walsh-Hadamard transform of n vectors of length d
 * (Sec. "Fast Walsh Hadamard": H_n = [[H_{n-1}, H_{n-1}], [H_{n-1}, -H_{n-1}]]).
 *   x     device, n x d float32, contiguous, 16-byte aligned when d >= 4
 *   n     number of vectors (>= 0)
 *   d     power of two, 1 <= d <= 2^20
 *   prec  MCK_FP32: float32 butterflies, any d; d <= 2^17 runs one pass over
 *         HBM (2^16 and 2^17 on thread-block clusters), larger d two.
 *         MCK_BF16 / MCK_FP16 / *_SPLIT: the Kronecker factorisation
 *         H_16 (x) H_16 (x) H_{d/256} on tensor cores (16-bit operands, the
 *         +-1 factor exact, FP32 accumulation; *_SPLIT rounds each operand
 *         as hi + lo to recover ~16 more bits) for d in {256, 512, 1024};
 *         for 1024 < d <= 2^20, H_d = H_{d/1024} (x) H_1024 with the tensor
 *         cores on every 1024-float block and FP32 column passes for the
 *         index bits above 10. Needs 256 <= d and n * d a multiple of 1024
 *         (MCK_EUNSUPPORTED / MCK_EINVAL otherwise). */
mck_status_t mck_fwht(float* x, int64_t n, int64_t d, int32_t prec, mck_stream_t stream);

/* How the FP32 transform runs at d = 2^16 and 2^17 (a tunable: every regime
 * gives bit-identical results; see paper_1702_08159_gb300/tune.py). */
typedef enum {
  MCK_FWHT_AUTO = 0,          /* the library's choice (MCK_FWHT_CLUSTER_2_15) */
  MCK_FWHT_CLUSTER_2_15 = 1,  /* one pass, a thread-block cluster of 2 or 4 blocks of 2^15 */
  MCK_FWHT_CLUSTER_2_14 = 2,  /* one pass, a cluster of 4 or 8 blocks of 2^14 */
  MCK_FWHT_TWO_PASS = 3       /* 2^15-float blocks, then a column pass over HBM */
} mck_fwht_regime_t;

/* mck_fwht with the regime for d = 2^16, 2^17 (prec must be MCK_FP32 there
 * when regime != MCK_FWHT_AUTO; at other d only MCK_FWHT_AUTO is accepted).
 * Errors as mck_fwht, plus MCK_EINVAL for an unknown or inapplicable regime. */
mck_status_t mck_fwht_ex(float* x, int64_t n, int64_t d, int32_t prec, int32_t regime,
                         mck_stream_t stream);

/* phi = features of n samples (Eq. etn:mckernel, Eq. etn:mcfeatures).
 *   x       device n x in_dim (ld ldx), 1 <= in_dim <= d; padded with zeros to d
 *   Cs, G   device E x d or NULL (plan tables)
 *   phi     device n x (2 E d), 16-byte aligned; row = E blocks of [cos | sin]
 * d <= 2^15 runs fused kernels (phi is the only output traffic). Above 2^15
 * the map runs in passes (signs, transform, gather with G, transform, Cs and
 * [cos | sin]) over stream-ordered scratch of at most 256 MiB, rows in
 * chunks. */
mck_status_t mck_features(mck_plan_t plan, const float* x, int64_t n, int64_t in_dim,
                          int64_t ldx, const float* Cs, const float* G, float* phi,
                          mck_stream_t stream);

/* ---- Host buffers ------------------------------------------------------------
 * Features of a batch held in HOST memory, written to host memory: the batch
 * moves in chunks of rows; each chunk's host-to-device copy, feature kernel
 * and device-to-host copy are queued on one of the pipe's streams, so the
 * copies of different chunks overlap one another and the kernels. A pipe owns
 * its streams and per-stream device buffers (chunk_rows x in_dim inputs,
 * chunk_rows x 2Ed features, and the multi-pass scratch above d = 2^15), made
 * once: calls allocate nothing. */
typedef struct mck_host_pipe_s* mck_host_pipe_t;
#define MCK_HOST_PIPE_MAX_STREAMS 16

/* Make a pipe for `plan` (which must outlive it) and inputs in_dim wide.
 *   chunk_rows  rows per chunk (>= 1); streams 1..MCK_HOST_PIPE_MAX_STREAMS.
 * Errors: MCK_EINVAL, MCK_ENOMEM (device buffers), MCK_ECUDA. */
mck_status_t mck_host_pipe_create(mck_host_pipe_t* out, mck_plan_t plan, int64_t in_dim,
                                  int64_t chunk_rows, int32_t streams);

/* phi = features of n samples, host to host, through the pipe.
 *   x     HOST n x in_dim float32 (ld ldx >= in_dim); pinned memory
 *         (cudaHostAlloc / cudaHostRegister) lets the copies run asynchronously
 *         and overlap the kernels; pageable memory works, with copies staged by
 *         the driver
 *   Cs, G DEVICE E x d or NULL (plan tables), as in mck_features
 *   phi   HOST n x 2Ed float32, the layout of mck_features
 * Stream-ordered: the pipe's streams start after the work queued on `stream`
 * so far, and `stream` waits for every chunk; synchronise `stream` before
 * reading phi. Calls on one pipe must not overlap (they share its buffers).
 * Host arrays are not extent-checked (their size is the caller's); a device
 * pointer returns MCK_EINVAL. */
mck_status_t mck_features_host(mck_host_pipe_t pipe, const float* x, int64_t n, int64_t ldx,
                               const float* Cs, const float* G, float* phi, mck_stream_t stream);

/* Release a pipe (synchronises its streams first). NULL is ignored. */
void mck_host_pipe_destroy(mck_host_pipe_t pipe);

/* mck_features with the two transforms in a chosen precision (the
 * tensor-core Kronecker-H16 transform of mck_fwht inside the feature map of
 * Eq. etn:mckernel; d = 1024 only, else MCK_EUNSUPPORTED):
 *   prec  MCK_FP32: mck_features itself. MCK_BF16 / MCK_FP16 / *_SPLIT: each H
 *         as the Kronecker factorisation H_4 (x) H_16 (x) H_16 with the two H16
 *         digits on the tensor cores (16-bit data operand, +-1 exact, FP32
 *         accumulation; *_SPLIT multiplies the hi and lo halves of the data)
 *         and the last two index bits as FP32 butterflies, in registers; the
 *         data is scaled per row by a power of two to keep it in fp16's range.
 *         Only the Pi gather goes through shared memory.
 * Accuracy against the FP64 oracle is stated in the tests (MCK_FP16_SPLIT
 * meets the FP32 bar of 1e-5 at the MNIST-shaped workloads; the unsplit forms
 * do not). Other arguments and errors as mck_features. */
mck_status_t mck_features_ex(mck_plan_t plan, const float* x, int64_t n, int64_t in_dim,
                             int64_t ldx, const float* Cs, const float* G, float* phi,
                             int32_t prec, mck_stream_t stream);

/* Gradients of sum(phi(x) * dphi) (the adjoint of mck_features, with H^T = H
 * and Pi^T = Pi^{-1}; the forward is recomputed, nothing is stored).
 * 32 <= d <= 2^20: fused kernels up to d = 1024, passes over stream-ordered
 * scratch (at most 256 MiB) above; MCK_EUNSUPPORTED below 32.
 *   dphi  device n x (2 E d)
 *   dx    device n x in_dim (ld ldx) or NULL
 *   dCs   device E x d or NULL: sum over samples of h * dz
 *   dG    device E x d or NULL: sum over samples of v * dw
 * Uses stream-ordered scratch memory of about 2 E d x 4 bytes per 8 samples. */
mck_status_t mck_features_backward(mck_plan_t plan, const float* x, int64_t n, int64_t in_dim,
                                   int64_t ldx, const float* Cs, const float* G,
                                   const float* dphi, float* dx, float* dCs, float* dG,
                                   mck_stream_t stream);

/* mck_features_backward plus the gradient with respect to B read as a real
 * diagonal (u0 = B x-hat, linear in B):
 *   dB    device E x d or NULL: sum over samples of x-hat * du0, with du0 the
 *         gradient reaching u0 (zero at k >= in_dim, where x-hat is padding)
 * With dB the scratch memory is 3 E d x 4 bytes per 8 samples. */
mck_status_t mck_features_backward_ex(mck_plan_t plan, const float* x, int64_t n,
                                      int64_t in_dim, int64_t ldx, const float* Cs,
                                      const float* G, const float* dphi, float* dx, float* dCs,
                                      float* dG, float* dB, mck_stream_t stream);

/* logits = phi(x) W^T + b without writing phi to memory (Sec. "Empirical
 * Analysis": softmax(W phi + b); the softmax itself is mck_softmax_xent).
 *   W        device num_classes x (2 E d)
 *   b        device num_classes or NULL (zero bias)
 *   logits   device n x num_classes
 * 1 <= num_classes <= MCK_MAX_CLASSES. Uses stream-ordered scratch memory of
 * at most n x E x num_classes floats for partial logits (none at d = 1024
 * when the batch has at least 8 rows per SM). Above d = 2^15 the features of
 * the rows in flight go to scratch (at most 256 MiB) before the contraction. */
mck_status_t mck_fused_logits(mck_plan_t plan, const float* x, int64_t n, int64_t in_dim,
                              int64_t ldx, const float* Cs, const float* G, const float* W,
                              const float* b, int32_t num_classes, float* logits,
                              mck_stream_t stream);

/* mck_fused_logits with the contraction W phi in a chosen precision (Sec.
 * "Empirical Analysis and Experiments": softmax(W phi + b); the tensor-core
 * split-precision contraction):
 *   prec  MCK_FP32: mck_fused_logits itself (FP32 FMA contraction, any d).
 *         MCK_FP16_SPLIT (d = 1024 only, else MCK_EUNSUPPORTED): the
 *         features are computed in FP32 as in mck_features and contracted on
 *         the tensor cores: each feature and each weight is written as
 *         hi + lo in fp16 (the weights of class c first scaled by a power of
 *         two so that their largest magnitude lies in [2^14, 2^15); exact,
 *         undone at the end), and hi.hi + hi.lo + lo.hi are accumulated in
 *         FP32. Each product then carries a relative error below ~2^-21;
 *         the tests hold the logits to the FP32 path's bar of 1e-4 against
 *         the FP64 oracle. Other precisions return MCK_EUNSUPPORTED.
 * Takes stream-ordered scratch for the split weights (E x 64 KiB, x 2 above
 * 8 classes) and, for batches with fewer 16-row tiles than resident blocks
 * (three per SM), n x (expansion chunks) x num_classes partial logits. Other arguments, results
 * and errors as mck_fused_logits. */
mck_status_t mck_fused_logits_ex(mck_plan_t plan, const float* x, int64_t n, int64_t in_dim,
                                 int64_t ldx, const float* Cs, const float* G, const float* W,
                                 const float* b, int32_t num_classes, float* logits,
                                 int32_t prec, mck_stream_t stream);

/* Capacity, in floats, of the fixed scratch used by mck_fused_logits_noalloc. */
#define MCK_NOALLOC_MAX_PARTIALS (1 << 22) /* 4,194,304 floats = 16 MiB per device */

/* mck_fused_logits without any memory allocation. (The paper has no
 * counterpart: this is a library convenience.) Same arguments and results as
 * mck_fused_logits. It is for callers that must not allocate device memory
 * while they run -- for example a serving loop that fixes its memory budget
 * at start-up and must not pay allocation latency or risk an out-of-memory
 * failure mid-request, or code that manages all device memory through its
 * own pool and forbids other allocations.
 *
 * Instead of stream-ordered scratch, the partial logits go to an array of
 * MCK_NOALLOC_MAX_PARTIALS floats (16 MiB) compiled into the library; each
 * GPU on which the library is used holds its own copy until the process
 * exits. How many partials a call needs depends on its shape: none at
 * d = 1024 when the batch has at least 8 rows per SM (the tile kernel writes
 * the logits directly; the 60000 x E = 16 x 10-class MNIST-shaped batch is
 * one such call), n x (expansion chunks) x num_classes for smaller batches at
 * d = 1024, and n x E x num_classes at every other d. A call that would need
 * more than the array holds returns MCK_EINVAL before any work is queued
 * (split the batch instead). The first call on a device looks up the
 * array's device address (with that device current) and caches it; make
 * that first call before any stream capture. The cached address belongs to
 * the device's current CUDA context: after cudaDeviceReset (or any teardown
 * of the primary context) every later call is invalid, as plans are. The
 * call performs no cudaMalloc or cudaFree and calls no allocating library
 * routine. All calls share the one array per device and every call fully
 * overwrites the part it uses, so nothing carries over from a previous call;
 * but calls whose work overlaps on the GPU (different streams, or different
 * threads) race on the array and must be serialised by the caller. */
mck_status_t mck_fused_logits_noalloc(mck_plan_t plan, const float* x, int64_t n, int64_t in_dim,
                                      int64_t ldx, const float* Cs, const float* G,
                                      const float* W, const float* b, int32_t num_classes,
                                      float* logits, mck_stream_t stream);

/* Gradients of sum(logits * dlogits) for mck_fused_logits: dx, dCs, dG, dW
 * (num_classes x 2Ed) and db (num_classes); any output may be NULL. */
mck_status_t mck_fused_logits_backward(mck_plan_t plan, const float* x, int64_t n,
                                       int64_t in_dim, int64_t ldx, const float* Cs,
                                       const float* G, const float* W, int32_t num_classes,
                                       const float* dlogits, float* dx, float* dCs, float* dG,
                                       float* dW, float* db, mck_stream_t stream);

/* mck_fused_logits_backward plus dB (device E x d or NULL), the gradient with
 * respect to B read as a real diagonal, as in mck_features_backward_ex. */
mck_status_t mck_fused_logits_backward_ex(mck_plan_t plan, const float* x, int64_t n,
                                          int64_t in_dim, int64_t ldx, const float* Cs,
                                          const float* G, const float* W, int32_t num_classes,
                                          const float* dlogits, float* dx, float* dCs,
                                          float* dG, float* dB, float* dW, float* db,
                                          mck_stream_t stream);

/* ---- Uneven batches in one persistent launch -------------------------------
 * A group is a prepared batch of vectors of different padded dimensions,
 * kernels and expansion counts (each vector uses the first E expansions of
 * its plan; Sec. "McKernel": expansions are i.i.d. instances of Z-hat). All
 * its work runs in ONE persistent kernel launch that takes units of work from
 * an atomic counter. Plans must outlive the group. */
typedef struct mck_group_s* mck_group_t;

typedef struct {
  int32_t plan;       /* index into the plans array given to mck_group_create */
  int32_t E;          /* expansions used: the plan's first E, 1 <= E <= the plan's E */
  int64_t in_dim;     /* input length, 1 <= in_dim <= the plan's d (zero padded to d) */
  int64_t x_offset;   /* element offset of the input vector in x */
  int64_t phi_offset; /* element offset of its 2*E*d features in phi; a multiple of 4 */
} mck_group_item_t;

/* Build the work list of a group (host work plus a small device upload;
 * synchronous). plans: host array of num_plans plans on one device with
 * 32 <= d <= 2^14. items: host array. x_len / phi_len: the element counts of
 * the x and phi arrays later passed to mck_group_features; every item must
 * fit inside them. grain: warp steps a warp takes from the work counter at a
 * time (0 picks the default, 2); a tunable, see mck_group_set_grain. Feature
 * layout of an item: E blocks of [cos (d) | sin (d)] at phi + phi_offset. */
mck_status_t mck_group_create(mck_group_t* out, const mck_plan_t* plans, int32_t num_plans,
                              const mck_group_item_t* items, int64_t num_items, int64_t x_len,
                              int64_t phi_len, int32_t grain);

/* Set the grain (1..64) used by later launches (a CUDA graph captured
 * earlier keeps the grain it was captured with). Host only. */
mck_status_t mck_group_set_grain(mck_group_t group, int32_t grain);

/* Sizes of the work list; any output may be NULL. num_units: the number of
 * phases (one per kind of work and d: block items of one d, or warp steps of
 * one d), each run to completion by all blocks before the next. */
mck_status_t mck_group_info(mck_group_t group, int64_t* num_units, int64_t* num_warp_steps,
                            int64_t* num_block_items, int32_t* grain);

/* Features of every item of the group: one memset of the work counters and
 * one persistent kernel launch on `stream`. Allocates nothing and does not
 * synchronise, so the call can be captured in a CUDA graph. x (x_len floats)
 * and phi (phi_len floats, 16-byte aligned) are device arrays. Calls on one
 * group must not overlap on the GPU (they share the work counters). */
mck_status_t mck_group_features(mck_group_t group, const float* x, float* phi,
                                mck_stream_t stream);

/* Release a group (synchronises its device first). NULL is ignored. */
void mck_group_destroy(mck_group_t group);

/* Mean softmax cross-entropy of logits (n x num_classes) against labels
 * (int32 in [0, num_classes)), the multi-class form of the logistic loss of
 * Eq. etn:loss. loss: device float[1] or NULL; dlogits: device n x
 * num_classes or NULL, (softmax - onehot)/n. A label outside the range makes
 * that row contribute 0 to loss and dlogits (a non-fatal data error). */
mck_status_t mck_softmax_xent(const float* logits, const int32_t* labels, int64_t n,
                              int32_t num_classes, float* loss, float* dlogits,
                              mck_stream_t stream);

/* Human-readable name of a status code (static storage). */
const char* mck_status_string(mck_status_t status);

/* Detail of the calling thread's most recent failure (static per thread). */
const char* mck_last_error(void);

#ifdef __cplusplus
}
#endif

#endif /* MCK_H */
