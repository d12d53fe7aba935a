/*
 * Plain FP32 CPU Fastfood feature map: the CPU comparison point for the GPU
 * kernels, written the way a straightforward multi-core CPU program computes
 * the method. It is neither the oracle (float64, in the paper's order, test
 * infrastructure) nor part of the GPU library, and shares no code with
 * either.
 *
 * Per sample and expansion e (Eq. etn:mckernel, Eq. etn:mcfeatures):
 *   u = H (B_e x-hat)      x-hat = x followed by zeros up to d
 *   v = G_e (Pi_e u)       (Pi u)_k = u_{pi_e(k)}
 *   z = Cs_e (H v)         Cs = C / (sigma sqrt d)
 *   phi = [cos z | sin z]
 * H is an iterative in-place radix-2 Walsh-Hadamard transform over one
 * d-float buffer (Sec. "Implementation of Fast Walsh Hadamard": the
 * transform runs in place, level by level, on data that stays in cache).
 * Samples are split over POSIX threads, one contiguous range each.
 *
 * The tables (B as +-1 floats, pi, G, Cs; E x d each, row-major) are inputs:
 * the caller builds them with whatever generator it trusts.
 */
#define _GNU_SOURCE
#include <math.h>
#include <pthread.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

typedef struct {
  const float* x;
  int64_t in_dim, ldx, d;
  int32_t E;
  const float* B;
  const uint32_t* perm;
  const float* G;
  const float* Cs;
  float* phi;
  int64_t out_rows; /* sample i is written to row i % out_rows of phi */
  int64_t row0, row1;
  int status;
} ff32_job;

/* In-place unnormalised Walsh-Hadamard transform of v[0..d), d = 2^L. */
static void fwht_inplace(float* v, int64_t d) {
  if (d >= 2)
    for (int64_t i = 0; i < d; i += 2) {
      const float a = v[i], b = v[i + 1];
      v[i] = a + b;
      v[i + 1] = a - b;
    }
  if (d >= 4)
    for (int64_t i = 0; i < d; i += 4) {
      const float a0 = v[i], a1 = v[i + 1], b0 = v[i + 2], b1 = v[i + 3];
      v[i] = a0 + b0;
      v[i + 1] = a1 + b1;
      v[i + 2] = a0 - b0;
      v[i + 3] = a1 - b1;
    }
  for (int64_t h = 4; h < d; h <<= 1)
    for (int64_t i = 0; i < d; i += 2 * h)
      for (int64_t j = i; j < i + h; ++j) {
        const float a = v[j], b = v[j + h];
        v[j] = a + b;
        v[j + h] = a - b;
      }
}

static void* ff32_worker(void* arg) {
  ff32_job* J = (ff32_job*)arg;
  const int64_t d = J->d;
  float* u = (float*)malloc(sizeof(float) * (size_t)d);
  float* v = (float*)malloc(sizeof(float) * (size_t)d);
  if (!u || !v) {
    free(u);
    free(v);
    J->status = -2;
    return NULL;
  }
  const int64_t F = 2 * (int64_t)J->E * d;
  for (int64_t i = J->row0; i < J->row1; ++i) {
    const float* xr = J->x + i * J->ldx;
    float* out = J->phi + (i % J->out_rows) * F;
    for (int32_t e = 0; e < J->E; ++e) {
      const float* Be = J->B + (int64_t)e * d;
      const uint32_t* pe = J->perm + (int64_t)e * d;
      const float* Ge = J->G + (int64_t)e * d;
      const float* Ce = J->Cs + (int64_t)e * d;
      for (int64_t k = 0; k < J->in_dim; ++k) u[k] = Be[k] * xr[k];
      for (int64_t k = J->in_dim; k < d; ++k) u[k] = 0.f;
      fwht_inplace(u, d);
      for (int64_t k = 0; k < d; ++k) v[k] = Ge[k] * u[pe[k]];
      fwht_inplace(v, d);
      float* oc = out + 2 * (int64_t)e * d;
      float* os = oc + d;
      for (int64_t k = 0; k < d; ++k) sincosf(Ce[k] * v[k], &os[k], &oc[k]);
    }
  }
  free(u);
  free(v);
  J->status = 0;
  return NULL;
}

/*
 * Features of n samples with `threads` POSIX threads (<= 0: one).
 *   x      n x in_dim float32, leading dimension ldx >= in_dim; 1 <= in_dim <= d
 *   d      power of two >= 1; E >= 1
 *   B, G, Cs  E x d float32; perm E x d uint32 (a permutation per row)
 *   phi    out_rows x 2Ed float32; sample i goes to row i % out_rows
 * Returns 0, -1 for a bad argument, -2 when memory or a thread could not be
 * had.
 */
int ff32_features(const float* x, int64_t n, int64_t in_dim, int64_t ldx, int64_t d, int32_t E,
                  const float* B, const uint32_t* perm, const float* G, const float* Cs,
                  float* phi, int64_t out_rows, int32_t threads) {
  if (n < 0 || d < 1 || (d & (d - 1)) || in_dim < 1 || in_dim > d || ldx < in_dim || E < 1 ||
      out_rows < 1)
    return -1;
  if (n == 0) return 0;
  if (!x || !B || !perm || !G || !Cs || !phi) return -1;
  int64_t T = threads < 1 ? 1 : threads;
  if (T > n) T = n;
  ff32_job* jobs = (ff32_job*)calloc((size_t)T, sizeof(ff32_job));
  pthread_t* tid = (pthread_t*)calloc((size_t)T, sizeof(pthread_t));
  if (!jobs || !tid) {
    free(jobs);
    free(tid);
    return -2;
  }
  char* created = (char*)calloc((size_t)T, 1);
  if (!created) {
    free(jobs);
    free(tid);
    return -2;
  }
  for (int64_t t = 0; t < T; ++t) {
    ff32_job* J = &jobs[t];
    J->x = x;
    J->in_dim = in_dim;
    J->ldx = ldx;
    J->d = d;
    J->E = E;
    J->B = B;
    J->perm = perm;
    J->G = G;
    J->Cs = Cs;
    J->phi = phi;
    J->out_rows = out_rows;
    J->row0 = n * t / T;
    J->row1 = n * (t + 1) / T;
    J->status = -2;
    /* the calling thread takes the last range, and any range whose thread
       could not be started */
    if (t + 1 < T && pthread_create(&tid[t], NULL, ff32_worker, J) == 0) created[t] = 1;
    else ff32_worker(J);
  }
  int status = 0;
  for (int64_t t = 0; t < T; ++t) {
    if (created[t]) pthread_join(tid[t], NULL);
    if (jobs[t].status != 0) status = jobs[t].status;
  }
  free(created);
  free(jobs);
  free(tid);
  return status;
}
