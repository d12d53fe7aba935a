// extern "C" entry points of libmck.so (declared in include/mck.h).
//
// Every call validates its arguments on the host before queuing device work:
// sizes, alignment, and that each array is device memory of the plan's
// device whose allocation contains the whole extent the call will touch
// (cuMemGetAddressRange). A wrong size or a host pointer therefore returns
// MCK_EINVAL instead of reaching a kernel.
#include <cuda.h>
#include <cuda_runtime.h>

#include <cmath>
#include <mutex>
#include <new>
#include <string>

#include "internal.h"

namespace mck {
namespace {

thread_local std::string g_last_error;

using AddressRangeFn = CUresult (*)(CUdeviceptr*, size_t*, CUdeviceptr);

AddressRangeFn address_range_fn() {
  static std::once_flag once;
  static AddressRangeFn fn = nullptr;
  std::call_once(once, [] {
    void* p = nullptr;
    cudaDriverEntryPointQueryResult q{};
    if (cudaGetDriverEntryPointByVersion("cuMemGetAddressRange", &p, 12000, cudaEnableDefault,
                                         &q) == cudaSuccess &&
        q == cudaDriverEntryPointSuccess)
      fn = reinterpret_cast<AddressRangeFn>(p);
    cudaGetLastError();
  });
  return fn;
}

int sm_count(int device) {
  static std::mutex mu;
  static int cache[64] = {0};
  std::lock_guard<std::mutex> lock(mu);
  if (device < 0 || device >= 64) return 1;
  if (!cache[device]) {
    int v = 0;
    if (cudaDeviceGetAttribute(&v, cudaDevAttrMultiProcessorCount, device) != cudaSuccess) {
      cudaGetLastError();
      v = 1;
    }
    cache[device] = v;
  }
  return cache[device];
}

// Sets the plan's device current for the duration of a call and restores
// the caller's device afterwards.
struct DeviceScope {
  int prev = -1;
  bool ok = true;
  explicit DeviceScope(int dev) {
    if (cudaGetDevice(&prev) != cudaSuccess) {
      cudaGetLastError();
      ok = false;
      return;
    }
    if (prev != dev && cudaSetDevice(dev) != cudaSuccess) {
      cudaGetLastError();
      ok = false;
    }
  }
  ~DeviceScope() {
    int cur = -1;
    if (prev >= 0 && cudaGetDevice(&cur) == cudaSuccess && cur != prev) cudaSetDevice(prev);
  }
};

bool is_pow2(int64_t v) { return v > 0 && (v & (v - 1)) == 0; }
int log2i(int64_t v) {
  int l = 0;
  while ((int64_t)1 << l < v) ++l;
  return l;
}

// `p` must be device memory on `device` whose allocation holds [p, p + bytes).
mck_status_t check_array(const void* p, int64_t bytes, int device, const char* name,
                         bool allow_null = false) {
  if (!p) {
    if (allow_null) return MCK_OK;
    return fail(MCK_EINVAL, std::string(name) + " is NULL");
  }
  if (bytes <= 0) return MCK_OK;
  cudaPointerAttributes at{};
  if (cudaPointerGetAttributes(&at, p) != cudaSuccess) {
    cudaGetLastError();
    return fail(MCK_EINVAL, std::string(name) + " is not a CUDA pointer");
  }
  if (at.type != cudaMemoryTypeDevice && at.type != cudaMemoryTypeManaged)
    return fail(MCK_EINVAL, std::string(name) + " is not device memory");
  if (at.type == cudaMemoryTypeDevice && at.device != device)
    return fail(MCK_EINVAL, std::string(name) + " lives on device " + std::to_string(at.device) +
                                ", the call runs on device " + std::to_string(device));
  if (AddressRangeFn fn = address_range_fn()) {
    CUdeviceptr base = 0;
    size_t size = 0;
    if (fn(&base, &size, (CUdeviceptr)p) == CUDA_SUCCESS) {
      const uint64_t lo = (uint64_t)(uintptr_t)p, end = (uint64_t)base + size;
      if (lo + (uint64_t)bytes > end)
        return fail(MCK_EINVAL, std::string(name) + ": " + std::to_string(bytes) +
                                    " bytes from this address run past the end of its allocation");
    }
  }
  return MCK_OK;
}

#define MCK_TRY(expr)                    \
  do {                                   \
    const mck_status_t _s = (expr);      \
    if (_s != MCK_OK) return _s;         \
  } while (0)

mck_status_t check_plan(const mck_plan_s* p) {
  if (!p) return fail(MCK_EINVAL, "plan is NULL");
  return MCK_OK;
}

mck_status_t check_x(const mck_plan_s* p, const float* x, int64_t n, int64_t in_dim, int64_t ldx) {
  if (n < 0) return fail(MCK_EINVAL, "n < 0");
  if (in_dim < 1 || in_dim > p->d) return fail(MCK_EINVAL, "in_dim must be in [1, d]");
  if (ldx < in_dim) return fail(MCK_EINVAL, "ldx < in_dim");
  if (n == 0) return MCK_OK;  // nothing is read; empty tensors may have no storage
  return check_array(x, 4 * ((n - 1) * ldx + in_dim), p->device, "x");
}

FeatureArgs feature_args(const mck_plan_s* p, const float* x, int64_t n, int64_t in_dim,
                         int64_t ldx, const float* Cs, const float* G) {
  FeatureArgs a{};
  a.x = x;
  a.n = n;
  a.in_dim = in_dim;
  a.ldx = ldx;
  a.B_bits = p->B_bits;
  a.perm = p->perm;
  a.G = G ? G : p->G;
  a.Cs = Cs ? Cs : p->Cs;
  a.permB = p->permB;
  a.GB = G ? nullptr : p->GB;  // an overriding G is read in natural order
  a.maskA = p->maskA;
  a.permS = p->permS;
  a.ubase = p->ubase;
  a.mmaMask = p->mmaMask;
  a.mmaG = G ? nullptr : p->mmaG;     // overriding tables are read in natural order
  a.mmaCs = Cs ? nullptr : p->mmaCs;
  a.mmaPerm = p->mmaPerm;
  a.mmaBase = p->mmaBase;
  a.rows_per_item = p->rows_per_item;
  a.staged = p->staged;
  a.E = p->E;
  a.L = p->L;
  a.num_sms = p->num_sms;
  return a;
}

mck_status_t check_tables(const mck_plan_s* p, const float* Cs, const float* G) {
  const int64_t bytes = 4 * p->d * p->E;
  MCK_TRY(check_array(Cs, bytes, p->device, "Cs", true));
  MCK_TRY(check_array(G, bytes, p->device, "G", true));
  if ((Cs && (uintptr_t)Cs % 16) || (G && (uintptr_t)G % 16))
    return fail(MCK_EINVAL, "Cs and G must be 16-byte aligned");
  return MCK_OK;
}

mck_status_t launched(cudaError_t err, const char* where) {
  return err == cudaSuccess ? MCK_OK : cuda_fail(err, where);
}

// The memory pool of a device that the calls' scratch comes from. The
// device's default pool hands unused memory back to the driver at every
// synchronisation (release threshold 0), so a call made after a synchronise
// would map its scratch anew each time; this pool keeps up to kScratchKeep
// bytes mapped between calls. Made on first use, with the device current (a
// process-wide setting of the default pool stays untouched); a context
// reset invalidates it, as it does plans. Null if it cannot be made: the
// scratch then comes from the default pool.
constexpr uint64_t kScratchKeep = 1ull << 30;
constexpr int kMaxDevices = 64;

cudaMemPool_t scratch_pool() {
  static std::mutex mu;
  static cudaMemPool_t pools[kMaxDevices] = {};
  static bool failed[kMaxDevices] = {};
  int device = 0;
  if (cudaGetDevice(&device) != cudaSuccess || device < 0 || device >= kMaxDevices) {
    cudaGetLastError();
    return nullptr;
  }
  std::lock_guard<std::mutex> lock(mu);
  if (!pools[device] && !failed[device]) {
    cudaMemPoolProps props{};
    props.allocType = cudaMemAllocationTypePinned;
    props.handleTypes = cudaMemHandleTypeNone;
    props.location.type = cudaMemLocationTypeDevice;
    props.location.id = device;
    cudaMemPool_t pool = nullptr;
    uint64_t keep = kScratchKeep;
    if (cudaMemPoolCreate(&pool, &props) != cudaSuccess ||
        cudaMemPoolSetAttribute(pool, cudaMemPoolAttrReleaseThreshold, &keep) != cudaSuccess) {
      cudaGetLastError();
      if (pool) cudaMemPoolDestroy(pool);
      failed[device] = true;
      return nullptr;
    }
    pools[device] = pool;
  }
  return pools[device];
}

// Stream-ordered scratch, freed on the same stream when the owner goes out of scope.
struct Scratch {
  void* ptr = nullptr;
  cudaStream_t s;
  explicit Scratch(cudaStream_t st) : s(st) {}
  mck_status_t alloc(size_t bytes) {
    if (bytes == 0) return MCK_OK;
    cudaMemPool_t pool = scratch_pool();
    const cudaError_t err = pool ? cudaMallocFromPoolAsync(&ptr, bytes, pool, s)
                                 : cudaMallocAsync(&ptr, bytes, s);
    if (err != cudaSuccess) {
      cudaGetLastError();
      ptr = nullptr;
      return fail(MCK_ENOMEM, "scratch allocation of " + std::to_string(bytes) + " bytes failed");
    }
    return MCK_OK;
  }
  ~Scratch() {
    if (ptr) cudaFreeAsync(ptr, s);
  }
};

}  // namespace

mck_status_t fail(mck_status_t s, const std::string& msg) {
  g_last_error = msg;
  return s;
}

mck_status_t check_device_array(const void* p, int64_t bytes, int device, const char* name) {
  return check_array(p, bytes, device, name);
}

mck_status_t cuda_fail(cudaError_t err, const char* where) {
  g_last_error = std::string(where) + ": " + cudaGetErrorName(err) + " (" + cudaGetErrorString(err) + ")";
  return MCK_ECUDA;
}

}  // namespace mck

using namespace mck;

extern "C" {

const char* mck_status_string(mck_status_t s) {
  switch (s) {
    case MCK_OK: return "MCK_OK";
    case MCK_EINVAL: return "MCK_EINVAL: invalid argument";
    case MCK_ENOMEM: return "MCK_ENOMEM: out of memory";
    case MCK_ECUDA: return "MCK_ECUDA: CUDA runtime error";
    case MCK_ETIMEOUT: return "MCK_ETIMEOUT: bounded wait expired";
    case MCK_EUNSUPPORTED: return "MCK_EUNSUPPORTED: not supported by this version";
  }
  return "unknown mck_status_t";
}

const char* mck_last_error(void) { return g_last_error.c_str(); }

mck_status_t mck_plan_ex(mck_plan_t* out, int64_t d, int32_t E, int32_t kernel, double sigma,
                         int32_t matern_t, uint64_t seed, int32_t device) {
  if (!out) return fail(MCK_EINVAL, "out is NULL");
  if (!is_pow2(d) || d < 2) return fail(MCK_EINVAL, "d must be a power of two >= 2");
  if (d > ((int64_t)1 << MCK_MAX_LOG2_D))
    return fail(MCK_EUNSUPPORTED, "plans support d <= 2^20");
  if (kernel == MCK_MATERN && d > ((int64_t)1 << MCK_MAX_LOG2_D_MATERN))
    return fail(MCK_EUNSUPPORTED, "Matern plans support d <= 2^15 (the ball sum draws t d^2 "
                                  "normals per expansion)");
  if (E < 1 || E > 65536) return fail(MCK_EINVAL, "E must be in [1, 65536]");
  if ((int64_t)E * d > ((int64_t)1 << 28)) return fail(MCK_EINVAL, "E * d must be <= 2^28");
  if (kernel != MCK_RBF && kernel != MCK_MATERN && kernel != MCK_LAPLACE) return fail(MCK_EINVAL, "unknown kernel");
  if (!(sigma > 0.0) || !std::isfinite(sigma)) return fail(MCK_EINVAL, "sigma must be finite and > 0");
  if (kernel == MCK_MATERN && (matern_t < 1 || matern_t > 4096))
    return fail(MCK_EINVAL, "Matern t must be in [1, 4096]");
  if (device < -1) return fail(MCK_EINVAL, "device must be >= -1");
  int ndev = 0;
  cudaError_t err = cudaGetDeviceCount(&ndev);
  if (err != cudaSuccess) {
    cudaGetLastError();
    return cuda_fail(err, "cudaGetDeviceCount");
  }
  if (device >= ndev) return fail(MCK_EINVAL, "no such device");
  if (device < 0 && (err = cudaGetDevice(&device)) != cudaSuccess) return cuda_fail(err, "cudaGetDevice");
  DeviceScope scope(device);
  if (!scope.ok) return fail(MCK_ECUDA, "cannot select the device");

  mck_plan_s* p = new (std::nothrow) mck_plan_s();
  if (!p) return fail(MCK_ENOMEM, "plan allocation failed");
  p->d = d;
  p->L = log2i(d);
  p->E = E;
  p->kernel = kernel;
  p->sigma = sigma;
  p->matern_t = kernel == MCK_MATERN ? matern_t : 0;
  p->seed = seed;
  p->device = device;
  p->num_sms = sm_count(device);
  p->words = (d + 31) / 32;
  const size_t n = (size_t)d * E;
  bool ok = cudaMalloc(&p->B_bits, sizeof(uint32_t) * p->words * E) == cudaSuccess &&
            cudaMalloc(&p->perm, sizeof(uint32_t) * n) == cudaSuccess &&
            cudaMalloc(&p->G, sizeof(float) * n) == cudaSuccess &&
            cudaMalloc(&p->Cs, sizeof(float) * n) == cudaSuccess;
  if (ok && p->L >= 5 && p->L <= 14) {
    const size_t T = (size_t)1 << (p->L - 5);
    ok = cudaMalloc(&p->permB, sizeof(uint32_t) * n) == cudaSuccess &&
         cudaMalloc(&p->GB, sizeof(float) * n) == cudaSuccess &&
         cudaMalloc(&p->maskA, sizeof(uint32_t) * T * E) == cudaSuccess;
  }
  if (ok && p->L == 10)
    ok = cudaMalloc(&p->permS, sizeof(uint32_t) * n / 2) == cudaSuccess &&
         cudaMalloc(&p->ubase, sizeof(uint32_t) * 32 * E) == cudaSuccess &&
         cudaMalloc(&p->mmaMask, sizeof(uint32_t) * 32 * E) == cudaSuccess &&
         cudaMalloc(&p->mmaG, sizeof(float) * n) == cudaSuccess &&
         cudaMalloc(&p->mmaCs, sizeof(float) * n) == cudaSuccess &&
         cudaMalloc(&p->mmaPerm, sizeof(uint32_t) * n / 2) == cudaSuccess &&
         cudaMalloc(&p->mmaBase, sizeof(uint32_t) * 32 * E) == cudaSuccess;
  if (!ok) {
    cudaGetLastError();
    mck_plan_destroy(p);
    return fail(MCK_ENOMEM, "plan table allocation failed");
  }
  cudaStream_t s = nullptr;
  if ((err = cudaStreamCreateWithFlags(&s, cudaStreamNonBlocking)) != cudaSuccess) {
    mck_plan_destroy(p);
    return cuda_fail(err, "cudaStreamCreate");
  }
  mck_status_t st = build_tables(p, s);
  cudaStreamDestroy(s);
  if (st == MCK_OK) st = build_skew_tables(p);
  if (st != MCK_OK) {
    mck_plan_destroy(p);
    return st;
  }
  *out = p;
  return MCK_OK;
}

mck_status_t mck_plan(mck_plan_t* out, int64_t d, int32_t E, int32_t kernel, double sigma,
                      uint64_t seed) {
  return mck_plan_ex(out, d, E, kernel, sigma, 40, seed, -1);
}

void mck_plan_destroy(mck_plan_t p) {
  if (!p) return;
  {
    DeviceScope scope(p->device);
    cudaDeviceSynchronize();
    cudaFree(p->B_bits);
    cudaFree(p->perm);
    cudaFree(p->G);
    cudaFree(p->Cs);
    cudaFree(p->permB);
    cudaFree(p->GB);
    cudaFree(p->maskA);
    cudaFree(p->permS);
    cudaFree(p->ubase);
    cudaFree(p->mmaMask);
    cudaFree(p->mmaG);
    cudaFree(p->mmaCs);
    cudaFree(p->mmaPerm);
    cudaFree(p->mmaBase);
    cudaGetLastError();
  }
  delete p;
}

mck_status_t mck_plan_info(mck_plan_t p, int64_t* d, int32_t* E, int32_t* kernel, double* sigma,
                           int32_t* matern_t, uint64_t* seed, int32_t* device) {
  MCK_TRY(check_plan(p));
  if (d) *d = p->d;
  if (E) *E = p->E;
  if (kernel) *kernel = p->kernel;
  if (sigma) *sigma = p->sigma;
  if (matern_t) *matern_t = p->matern_t;
  if (seed) *seed = p->seed;
  if (device) *device = p->device;
  return MCK_OK;
}

mck_status_t mck_plan_set_launch(mck_plan_t p, int32_t rows_per_item, int32_t staged) {
  MCK_TRY(check_plan(p));
  if (staged < -1 || staged > 1) return fail(MCK_EINVAL, "staged must be -1, 0 or 1");
  if (p->L >= 5 && p->L <= 10) {
    const int T = 1 << (p->L - 5), vpw = 32 / T, spi = vpw >= 4 ? vpw : 4;
    if (rows_per_item != 0 && rows_per_item != vpw && rows_per_item != spi)
      return fail(MCK_EINVAL, "rows_per_item at this d must be 0, " + std::to_string(vpw) +
                                  " or " + std::to_string(spi));
    if (staged != -1) return fail(MCK_EINVAL, "staging applies to 2^11 <= d <= 2^14 only");
  } else if (p->L >= 11 && p->L <= 14) {
    if (rows_per_item != 0 && rows_per_item != 1 && rows_per_item != 2 && rows_per_item != 4)
      return fail(MCK_EINVAL, "rows_per_item at this d must be 0, 1, 2 or 4");
  } else if (rows_per_item != 0 || staged != -1) {
    return fail(MCK_EINVAL, "this d has one launch shape (rows_per_item 0, staged -1)");
  }
  p->rows_per_item = rows_per_item;
  p->staged = staged;
  return MCK_OK;
}

mck_status_t mck_plan_get_launch(mck_plan_t p, int32_t* rows_per_item, int32_t* staged) {
  MCK_TRY(check_plan(p));
  if (rows_per_item) *rows_per_item = p->rows_per_item;
  if (staged) *staged = p->staged;
  return MCK_OK;
}

mck_status_t mck_plan_tables(mck_plan_t p, uint32_t* B_bits, uint32_t* perm, float* G, float* Cs) {
  MCK_TRY(check_plan(p));
  DeviceScope scope(p->device);
  const size_t n = (size_t)p->d * p->E;
  cudaError_t err = cudaSuccess;
  if (B_bits && err == cudaSuccess)
    err = cudaMemcpy(B_bits, p->B_bits, sizeof(uint32_t) * p->words * p->E, cudaMemcpyDeviceToHost);
  if (perm && err == cudaSuccess)
    err = cudaMemcpy(perm, p->perm, sizeof(uint32_t) * n, cudaMemcpyDeviceToHost);
  if (G && err == cudaSuccess) err = cudaMemcpy(G, p->G, sizeof(float) * n, cudaMemcpyDeviceToHost);
  if (Cs && err == cudaSuccess) err = cudaMemcpy(Cs, p->Cs, sizeof(float) * n, cudaMemcpyDeviceToHost);
  return launched(err, "mck_plan_tables");
}

mck_status_t mck_fwht(float* x, int64_t n, int64_t d, int32_t prec, mck_stream_t stream) {
  return mck_fwht_ex(x, n, d, prec, MCK_FWHT_AUTO, stream);
}

mck_status_t mck_fwht_ex(float* x, int64_t n, int64_t d, int32_t prec, int32_t regime,
                         mck_stream_t stream) {
  if (prec < MCK_FP32 || prec > MCK_FP16_SPLIT) return fail(MCK_EUNSUPPORTED, "unknown precision");
  if (regime < MCK_FWHT_AUTO || regime > MCK_FWHT_TWO_PASS) return fail(MCK_EINVAL, "unknown regime");
  if (regime != MCK_FWHT_AUTO && (prec != MCK_FP32 || (d != (1 << 16) && d != (1 << 17))))
    return fail(MCK_EINVAL, "a transform regime can be chosen only for FP32 at d = 2^16 or 2^17");
  if (!is_pow2(d)) return fail(MCK_EINVAL, "d must be a power of two");
  if (prec != MCK_FP32 && !fwht_mma_supported(log2i(d)))
    return fail(MCK_EUNSUPPORTED, "the tensor-core transform supports 256 <= d <= 2^20");
  if (prec != MCK_FP32 && ((n * d) & 1023))
    return fail(MCK_EINVAL, "the tensor-core transform needs n * d to be a multiple of 1024");
  if (d > ((int64_t)1 << MCK_MAX_LOG2_D_FWHT)) return fail(MCK_EUNSUPPORTED, "d must be <= 2^20");
  if (n < 0) return fail(MCK_EINVAL, "n < 0");
  if (n == 0 || d == 1) return MCK_OK;  // nothing to transform
  if (!x) return fail(MCK_EINVAL, "x is NULL");
  if (d >= 4 && (uintptr_t)x % 16) return fail(MCK_EINVAL, "x must be 16-byte aligned");
  int device = 0;
  cudaError_t err = cudaGetDevice(&device);
  if (err != cudaSuccess) return cuda_fail(err, "cudaGetDevice");
  MCK_TRY(check_array(x, 4 * n * d, device, "x"));
  if (prec != MCK_FP32)
    return launched(launch_fwht_mma(x, n, log2i(d), prec, sm_count(device), (cudaStream_t)stream),
                    "mck_fwht");
  return launched(launch_fwht(x, n, log2i(d), sm_count(device), (cudaStream_t)stream, regime),
                  "mck_fwht");
}

mck_status_t mck_features(mck_plan_t p, const float* x, int64_t n, int64_t in_dim, int64_t ldx,
                          const float* Cs, const float* G, float* phi, mck_stream_t stream) {
  MCK_TRY(check_plan(p));
  DeviceScope scope(p->device);
  MCK_TRY(check_x(p, x, n, in_dim, ldx));
  MCK_TRY(check_tables(p, Cs, G));
  const int64_t F = 2 * p->E * p->d;
  if (n == 0) return MCK_OK;
  MCK_TRY(check_array(phi, 4 * n * F, p->device, "phi"));
  if (p->d >= 4 && (uintptr_t)phi % 16) return fail(MCK_EINVAL, "phi must be 16-byte aligned");
  cudaStream_t s = (cudaStream_t)stream;
  if (p->L > 15) {  // multi-pass over a scratch of the rows in flight
    Scratch sc(s);
    MCK_TRY(sc.alloc(sizeof(float) * (size_t)multipass_scratch_floats(p->L, n, p->E, 0, false)));
    return launched(launch_features_multipass(feature_args(p, x, n, in_dim, ldx, Cs, G), phi,
                                              nullptr, nullptr, 0, nullptr, (float*)sc.ptr, s),
                    "mck_features");
  }
  return launched(launch_features(feature_args(p, x, n, in_dim, ldx, Cs, G), phi, s),
                  "mck_features");
}

mck_status_t mck_features_ex(mck_plan_t p, const float* x, int64_t n, int64_t in_dim, int64_t ldx,
                             const float* Cs, const float* G, float* phi, int32_t prec,
                             mck_stream_t stream) {
  if (prec == MCK_FP32) return mck_features(p, x, n, in_dim, ldx, Cs, G, phi, stream);
  MCK_TRY(check_plan(p));
  if (prec < MCK_BF16 || prec > MCK_FP16_SPLIT) return fail(MCK_EUNSUPPORTED, "unknown precision");
  if (p->L != 10) return fail(MCK_EUNSUPPORTED, "tensor-core features are built for d = 1024");
  DeviceScope scope(p->device);
  MCK_TRY(check_x(p, x, n, in_dim, ldx));
  MCK_TRY(check_tables(p, Cs, G));
  const int64_t F = 2 * p->E * p->d;
  if (n == 0) return MCK_OK;
  MCK_TRY(check_array(phi, 4 * n * F, p->device, "phi"));
  if ((uintptr_t)phi % 16) return fail(MCK_EINVAL, "phi must be 16-byte aligned");
  return launched(launch_features_mma(feature_args(p, x, n, in_dim, ldx, Cs, G), phi, prec,
                                      (cudaStream_t)stream),
                  "mck_features_ex");
}

static mck_status_t run_backward(mck_plan_s* p, BackwardArgs b, cudaStream_t s, const char* who) {
  const int64_t n = b.f.n;
  if (n == 0) return MCK_OK;
  if (p->L > 10) {  // multi-pass adjoint
    Scratch sc(s);
    MCK_TRY(sc.alloc(sizeof(float) * (size_t)multipass_scratch_floats(p->L, n, p->E, 0, true)));
    return launched(launch_backward_multipass(b, (float*)sc.ptr, s), who);
  }
  const bool params = b.dCs || b.dG || b.dB || b.phi_out;
  const int64_t np = params ? backward_partials(p->L, n, p->E, p->num_sms) : 0;
  Scratch part(s);
  MCK_TRY(part.alloc(sizeof(float) * (size_t)np * (b.dB ? 3 : 2) * p->d));
  return launched(launch_backward(b, (float*)part.ptr, np, s), who);
}

mck_status_t mck_features_backward_ex(mck_plan_t p, const float* x, int64_t n, int64_t in_dim,
                                      int64_t ldx, const float* Cs, const float* G,
                                      const float* dphi, float* dx, float* dCs, float* dG,
                                      float* dB, mck_stream_t stream) {
  MCK_TRY(check_plan(p));
  if (p->L < 5) return fail(MCK_EUNSUPPORTED, "the adjoint supports 32 <= d <= 2^20");
  DeviceScope scope(p->device);
  MCK_TRY(check_x(p, x, n, in_dim, ldx));
  MCK_TRY(check_tables(p, Cs, G));
  const int64_t F = 2 * p->E * p->d, tb = 4 * p->E * p->d;
  MCK_TRY(check_array(dCs, tb, p->device, "dCs", true));
  MCK_TRY(check_array(dG, tb, p->device, "dG", true));
  MCK_TRY(check_array(dB, tb, p->device, "dB", true));
  if (n == 0) {  // sums over an empty batch are zero
    cudaError_t err = cudaSuccess;
    if (dCs) err = cudaMemsetAsync(dCs, 0, tb, (cudaStream_t)stream);
    if (dG && err == cudaSuccess) err = cudaMemsetAsync(dG, 0, tb, (cudaStream_t)stream);
    if (dB && err == cudaSuccess) err = cudaMemsetAsync(dB, 0, tb, (cudaStream_t)stream);
    return launched(err, "mck_features_backward");
  }
  MCK_TRY(check_array(dphi, 4 * n * F, p->device, "dphi"));
  if ((uintptr_t)dphi % 16) return fail(MCK_EINVAL, "dphi must be 16-byte aligned");
  MCK_TRY(check_array(dx, 4 * ((n - 1) * ldx + in_dim), p->device, "dx", true));
  BackwardArgs b{};
  b.f = feature_args(p, x, n, in_dim, ldx, Cs, G);
  b.dphi = dphi;
  b.dx = dx;
  b.dCs = dCs;
  b.dG = dG;
  b.dB = dB;
  return run_backward(p, b, (cudaStream_t)stream, "mck_features_backward");
}

mck_status_t mck_features_backward(mck_plan_t p, const float* x, int64_t n, int64_t in_dim,
                                   int64_t ldx, const float* Cs, const float* G, const float* dphi,
                                   float* dx, float* dCs, float* dG, mck_stream_t stream) {
  return mck_features_backward_ex(p, x, n, in_dim, ldx, Cs, G, dphi, dx, dCs, dG, nullptr, stream);
}

mck_status_t mck_fused_logits(mck_plan_t p, const float* x, int64_t n, int64_t in_dim, int64_t ldx,
                              const float* Cs, const float* G, const float* W, const float* b,
                              int32_t C, float* logits, mck_stream_t stream) {
  MCK_TRY(check_plan(p));
  if (C < 1 || C > MCK_MAX_CLASSES) return fail(MCK_EINVAL, "num_classes must be in [1, 16]");
  DeviceScope scope(p->device);
  MCK_TRY(check_x(p, x, n, in_dim, ldx));
  MCK_TRY(check_tables(p, Cs, G));
  const int64_t F = 2 * p->E * p->d;
  MCK_TRY(check_array(W, 4 * C * F, p->device, "W"));
  if (p->d >= 4 && (uintptr_t)W % 16) return fail(MCK_EINVAL, "W must be 16-byte aligned");
  MCK_TRY(check_array(b, 4 * C, p->device, "b", true));
  if (n == 0) return MCK_OK;
  MCK_TRY(check_array(logits, 4 * n * C, p->device, "logits"));
  cudaStream_t s = (cudaStream_t)stream;
  Scratch part(s);
  const int64_t nparts = logits_scratch_floats(p->L, n, p->E, C, p->num_sms);
  if (nparts > 0) MCK_TRY(part.alloc(sizeof(float) * (size_t)nparts));
  return launched(launch_logits(feature_args(p, x, n, in_dim, ldx, Cs, G), W, b, C,
                                (float*)part.ptr, logits, s),
                  "mck_fused_logits");
}

mck_status_t mck_fused_logits_ex(mck_plan_t p, const float* x, int64_t n, int64_t in_dim,
                                 int64_t ldx, const float* Cs, const float* G, const float* W,
                                 const float* b, int32_t C, float* logits, int32_t prec,
                                 mck_stream_t stream) {
  if (prec == MCK_FP32) return mck_fused_logits(p, x, n, in_dim, ldx, Cs, G, W, b, C, logits, stream);
  MCK_TRY(check_plan(p));
  if (prec != MCK_FP16_SPLIT)
    return fail(MCK_EUNSUPPORTED, "the tensor-core contraction is built for MCK_FP16_SPLIT");
  if (p->L != 10) return fail(MCK_EUNSUPPORTED, "the tensor-core contraction is built for d = 1024");
  if (C < 1 || C > MCK_MAX_CLASSES) return fail(MCK_EINVAL, "num_classes must be in [1, 16]");
  DeviceScope scope(p->device);
  MCK_TRY(check_x(p, x, n, in_dim, ldx));
  MCK_TRY(check_tables(p, Cs, G));
  const int64_t F = 2 * p->E * p->d;
  MCK_TRY(check_array(W, 4 * C * F, p->device, "W"));
  if ((uintptr_t)W % 16) return fail(MCK_EINVAL, "W must be 16-byte aligned");
  MCK_TRY(check_array(b, 4 * C, p->device, "b", true));
  if (n == 0) return MCK_OK;
  MCK_TRY(check_array(logits, 4 * n * C, p->device, "logits"));
  cudaStream_t s = (cudaStream_t)stream;
  Scratch sc(s);
  MCK_TRY(sc.alloc(sizeof(float) * (size_t)logits_mma_scratch_floats(n, p->E, C, p->num_sms)));
  return launched(launch_logits_mma(feature_args(p, x, n, in_dim, ldx, Cs, G), W, b, C,
                                    (float*)sc.ptr, logits, s),
                  "mck_fused_logits_ex");
}

mck_status_t mck_fused_logits_backward_ex(mck_plan_t p, const float* x, int64_t n,
                                          int64_t in_dim, int64_t ldx, const float* Cs,
                                          const float* G, const float* W, int32_t C,
                                          const float* dlogits, float* dx, float* dCs, float* dG,
                                          float* dB, float* dW, float* db, mck_stream_t stream) {
  MCK_TRY(check_plan(p));
  if (p->L < 5) return fail(MCK_EUNSUPPORTED, "the adjoint supports 32 <= d <= 2^20");
  if (C < 1 || C > MCK_MAX_CLASSES) return fail(MCK_EINVAL, "num_classes must be in [1, 16]");
  DeviceScope scope(p->device);
  MCK_TRY(check_x(p, x, n, in_dim, ldx));
  MCK_TRY(check_tables(p, Cs, G));
  const int64_t F = 2 * p->E * p->d, tb = 4 * p->E * p->d;
  MCK_TRY(check_array(W, 4 * C * F, p->device, "W"));
  if ((uintptr_t)W % 16) return fail(MCK_EINVAL, "W must be 16-byte aligned");
  MCK_TRY(check_array(dCs, tb, p->device, "dCs", true));
  MCK_TRY(check_array(dG, tb, p->device, "dG", true));
  MCK_TRY(check_array(dB, tb, p->device, "dB", true));
  MCK_TRY(check_array(dW, 4 * C * F, p->device, "dW", true));
  MCK_TRY(check_array(db, 4 * C, p->device, "db", true));
  cudaStream_t s = (cudaStream_t)stream;
  if (n == 0) {
    // Gradients of an empty batch are zero.
    cudaError_t err = cudaSuccess;
    if (dCs) err = cudaMemsetAsync(dCs, 0, tb, s);
    if (dG && err == cudaSuccess) err = cudaMemsetAsync(dG, 0, tb, s);
    if (dB && err == cudaSuccess) err = cudaMemsetAsync(dB, 0, tb, s);
    if (dW && err == cudaSuccess) err = cudaMemsetAsync(dW, 0, 4 * C * F, s);
    if (db && err == cudaSuccess) err = cudaMemsetAsync(db, 0, 4 * C, s);
    return launched(err, "mck_fused_logits_backward");
  }
  MCK_TRY(check_array(dlogits, 4 * n * C, p->device, "dlogits"));
  MCK_TRY(check_array(dx, 4 * ((n - 1) * ldx + in_dim), p->device, "dx", true));
  Scratch phi(s);
  if (dW) MCK_TRY(phi.alloc(sizeof(float) * (size_t)n * F));
  BackwardArgs b{};
  b.f = feature_args(p, x, n, in_dim, ldx, Cs, G);
  b.W = W;
  b.dlogits = dlogits;
  b.C = C;
  b.phi_out = (float*)phi.ptr;
  b.dx = dx;
  b.dCs = dCs;
  b.dG = dG;
  b.dB = dB;
  MCK_TRY(run_backward(p, b, s, "mck_fused_logits_backward"));
  return launched(launch_logit_weight_grads(dlogits, (const float*)phi.ptr, n, C, F, dW, db, s),
                  "mck_fused_logits_backward");
}

mck_status_t mck_fused_logits_backward(mck_plan_t p, const float* x, int64_t n, int64_t in_dim,
                                       int64_t ldx, const float* Cs, const float* G, const float* W,
                                       int32_t C, const float* dlogits, float* dx, float* dCs,
                                       float* dG, float* dW, float* db, mck_stream_t stream) {
  return mck_fused_logits_backward_ex(p, x, n, in_dim, ldx, Cs, G, W, C, dlogits, dx, dCs, dG,
                                      nullptr, dW, db, stream);
}

mck_status_t mck_plan_set_signs(mck_plan_t p, const float* B, mck_stream_t stream) {
  MCK_TRY(check_plan(p));
  DeviceScope scope(p->device);
  MCK_TRY(check_array(B, 4 * p->E * p->d, p->device, "B"));
  return launched(set_signs(p, B, (cudaStream_t)stream), "mck_plan_set_signs");
}

mck_status_t mck_softmax_xent(const float* logits, const int32_t* labels, int64_t n, int32_t C,
                              float* loss, float* dlogits, mck_stream_t stream) {
  if (n < 0) return fail(MCK_EINVAL, "n < 0");
  if (C < 1) return fail(MCK_EINVAL, "num_classes must be >= 1");
  int device = 0;
  cudaError_t err = cudaGetDevice(&device);
  if (err != cudaSuccess) return cuda_fail(err, "cudaGetDevice");
  MCK_TRY(check_array(loss, 4, device, "loss", true));
  if (n == 0) {
    if (loss) return launched(cudaMemsetAsync(loss, 0, 4, (cudaStream_t)stream), "mck_softmax_xent");
    return MCK_OK;
  }
  MCK_TRY(check_array(logits, 4 * n * C, device, "logits"));
  MCK_TRY(check_array(labels, 4 * n, device, "labels"));
  MCK_TRY(check_array(dlogits, 4 * n * C, device, "dlogits", true));
  return launched(launch_softmax_xent(logits, labels, n, C, loss, dlogits, (cudaStream_t)stream),
                  "mck_softmax_xent");
}

}  // extern "C"

// ---------------------------------------------------------------------------
// Allocation-free fused logits.
//
// mck_fused_logits takes n x E x C floats of stream-ordered scratch for the
// per-(sample, expansion) partial logits. This variant keeps that scratch in
// a fixed array compiled into the library instead, so a call performs no
// allocation at all. The array lives in device memory of every GPU on which
// the library's code is loaded, for the life of the process.
// ---------------------------------------------------------------------------
namespace {

__device__ __align__(256) float g_noalloc_partials[MCK_NOALLOC_MAX_PARTIALS];

std::mutex g_noalloc_mu;
float* g_noalloc_ptr[64] = {};

// Device address of the fixed scratch on `device` (which must be current).
// In host code the array's name is only a host-side handle, so the address
// is looked up once per device and cached.
mck_status_t noalloc_scratch(int device, float** out) {
  if (device < 0 || device >= 64) return fail(MCK_EINVAL, "device index out of range");
  std::lock_guard<std::mutex> lock(g_noalloc_mu);
  if (!g_noalloc_ptr[device]) {
    void* p = nullptr;
    const cudaError_t err = cudaGetSymbolAddress(&p, g_noalloc_partials);
    if (err != cudaSuccess) {
      cudaGetLastError();
      return cuda_fail(err, "cudaGetSymbolAddress(fixed logits scratch)");
    }
    g_noalloc_ptr[device] = static_cast<float*>(p);
  }
  *out = g_noalloc_ptr[device];
  return MCK_OK;
}

}  // namespace

extern "C" mck_status_t mck_fused_logits_noalloc(mck_plan_t p, const float* x, int64_t n,
                                                 int64_t in_dim, int64_t ldx, const float* Cs,
                                                 const float* G, const float* W, const float* b,
                                                 int32_t C, float* logits, mck_stream_t stream) {
  MCK_TRY(check_plan(p));
  if (C < 1 || C > MCK_MAX_CLASSES) return fail(MCK_EINVAL, "num_classes must be in [1, 16]");
  // The kernels pick the amount of partial logits from the batch shape: none
  // at d = 1024 with at least one 8-row tile per SM, n x (chunks of E) x C for
  // smaller batches there, n x E x C at other d.
  const int64_t need = n > 0 ? logits_scratch_floats(p->L, n, p->E, C, p->num_sms) : 0;
  if (need > (int64_t)MCK_NOALLOC_MAX_PARTIALS)
    return fail(MCK_EINVAL, std::to_string(need) +
                                " partial logits exceed the fixed scratch of " +
                                std::to_string((int64_t)MCK_NOALLOC_MAX_PARTIALS) +
                                " floats (split the batch)");
  DeviceScope scope(p->device);
  if (!scope.ok) return fail(MCK_ECUDA, "cannot select the plan's device");
  MCK_TRY(check_x(p, x, n, in_dim, ldx));
  MCK_TRY(check_tables(p, Cs, G));
  const int64_t F = 2 * p->E * p->d;
  MCK_TRY(check_array(W, 4 * C * F, p->device, "W"));
  if (p->d >= 4 && (uintptr_t)W % 16) return fail(MCK_EINVAL, "W must be 16-byte aligned");
  MCK_TRY(check_array(b, 4 * C, p->device, "b", true));
  float* scratch = nullptr;
  MCK_TRY(noalloc_scratch(p->device, &scratch));
  if (n == 0) return MCK_OK;
  MCK_TRY(check_array(logits, 4 * n * C, p->device, "logits"));
  // Every partial read by the reduction is written first by the feature
  // kernel of this call, so the array needs no clearing between calls.
  return launched(launch_logits(feature_args(p, x, n, in_dim, ldx, Cs, G), W, b, C, scratch,
                                logits, (cudaStream_t)stream),
                  "mck_fused_logits_noalloc");
}

// ---------------------------------------------------------------------------
// Host-buffer features: chunks of rows through per-stream device buffers.
// ---------------------------------------------------------------------------
struct mck_host_pipe_s {
  mck_plan_s* plan = nullptr;
  int64_t in_dim = 0, rows = 0, scratch_floats = 0;
  int ns = 0;
  cudaStream_t st[MCK_HOST_PIPE_MAX_STREAMS] = {};
  cudaEvent_t done[MCK_HOST_PIPE_MAX_STREAMS] = {};
  cudaEvent_t start = nullptr;
  float* xd[MCK_HOST_PIPE_MAX_STREAMS] = {};
  float* pd[MCK_HOST_PIPE_MAX_STREAMS] = {};
  float* sc[MCK_HOST_PIPE_MAX_STREAMS] = {};
};

extern "C" void mck_host_pipe_destroy(mck_host_pipe_t h) {
  if (!h) return;
  {
    DeviceScope scope(h->plan->device);
    for (int i = 0; i < h->ns; ++i) {
      if (h->st[i]) cudaStreamSynchronize(h->st[i]);
      cudaFree(h->xd[i]);
      cudaFree(h->pd[i]);
      cudaFree(h->sc[i]);
      if (h->done[i]) cudaEventDestroy(h->done[i]);
      if (h->st[i]) cudaStreamDestroy(h->st[i]);
    }
    if (h->start) cudaEventDestroy(h->start);
    cudaGetLastError();
  }
  delete h;
}

extern "C" mck_status_t mck_host_pipe_create(mck_host_pipe_t* out, mck_plan_t p, int64_t in_dim,
                                             int64_t chunk_rows, int32_t streams) {
  if (!out) return fail(MCK_EINVAL, "out is NULL");
  MCK_TRY(check_plan(p));
  if (in_dim < 1 || in_dim > p->d) return fail(MCK_EINVAL, "in_dim must be in [1, d]");
  if (chunk_rows < 1) return fail(MCK_EINVAL, "chunk_rows must be >= 1");
  if (streams < 1 || streams > MCK_HOST_PIPE_MAX_STREAMS)
    return fail(MCK_EINVAL, "streams must be in [1, MCK_HOST_PIPE_MAX_STREAMS]");
  DeviceScope scope(p->device);
  if (!scope.ok) return fail(MCK_ECUDA, "cannot select the plan's device");
  mck_host_pipe_s* h = new (std::nothrow) mck_host_pipe_s();
  if (!h) return fail(MCK_ENOMEM, "pipe allocation failed");
  h->plan = p;
  h->in_dim = in_dim;
  h->rows = chunk_rows;
  h->ns = streams;
  const int64_t F = 2 * p->E * p->d;
  h->scratch_floats = p->L > 15 ? multipass_scratch_floats(p->L, chunk_rows, p->E, 0, false) : 0;
  bool ok = cudaEventCreateWithFlags(&h->start, cudaEventDisableTiming) == cudaSuccess;
  for (int i = 0; ok && i < streams; ++i) {
    ok = cudaStreamCreateWithFlags(&h->st[i], cudaStreamNonBlocking) == cudaSuccess &&
         cudaEventCreateWithFlags(&h->done[i], cudaEventDisableTiming) == cudaSuccess &&
         cudaMalloc(&h->xd[i], sizeof(float) * (size_t)(chunk_rows * in_dim)) == cudaSuccess &&
         cudaMalloc(&h->pd[i], sizeof(float) * (size_t)(chunk_rows * F)) == cudaSuccess &&
         (h->scratch_floats == 0 ||
          cudaMalloc(&h->sc[i], sizeof(float) * (size_t)h->scratch_floats) == cudaSuccess);
  }
  if (!ok) {
    cudaGetLastError();
    mck_host_pipe_destroy(h);
    return fail(MCK_ENOMEM, "pipe streams or device buffers could not be made");
  }
  *out = h;
  return MCK_OK;
}

// Host memory (pinned or pageable), not device or managed memory.
static mck_status_t check_host(const void* ptr, const char* name) {
  if (!ptr) return fail(MCK_EINVAL, std::string(name) + " is NULL");
  cudaPointerAttributes at{};
  if (cudaPointerGetAttributes(&at, ptr) != cudaSuccess) {
    cudaGetLastError();
    return MCK_OK;  // not known to CUDA: pageable host memory
  }
  if (at.type == cudaMemoryTypeDevice || at.type == cudaMemoryTypeManaged)
    return fail(MCK_EINVAL, std::string(name) + " is device memory; mck_features takes device arrays");
  return MCK_OK;
}

extern "C" mck_status_t mck_features_host(mck_host_pipe_t h, const float* x, int64_t n, int64_t ldx,
                                          const float* Cs, const float* G, float* phi,
                                          mck_stream_t stream) {
  if (!h) return fail(MCK_EINVAL, "pipe is NULL");
  mck_plan_s* p = h->plan;
  if (n < 0) return fail(MCK_EINVAL, "n < 0");
  if (ldx < h->in_dim) return fail(MCK_EINVAL, "ldx < in_dim");
  if (n == 0) return MCK_OK;
  DeviceScope scope(p->device);
  if (!scope.ok) return fail(MCK_ECUDA, "cannot select the plan's device");
  MCK_TRY(check_host(x, "x"));
  MCK_TRY(check_host(phi, "phi"));
  MCK_TRY(check_tables(p, Cs, G));
  cudaStream_t s = (cudaStream_t)stream;
  const int64_t F = 2 * p->E * p->d;
  const int64_t chunks = (n + h->rows - 1) / h->rows;
  const int k = (int)std::min<int64_t>(h->ns, chunks);
  cudaError_t err = cudaEventRecord(h->start, s);
  for (int i = 0; err == cudaSuccess && i < k; ++i) err = cudaStreamWaitEvent(h->st[i], h->start, 0);
  for (int64_t c = 0; err == cudaSuccess && c < chunks; ++c) {
    const int i = (int)(c % k);
    const int64_t a = c * h->rows, rows = std::min<int64_t>(h->rows, n - a);
    cudaStream_t si = h->st[i];
    err = ldx == h->in_dim
              ? cudaMemcpyAsync(h->xd[i], x + a * ldx, sizeof(float) * rows * ldx,
                                cudaMemcpyHostToDevice, si)
              : cudaMemcpy2DAsync(h->xd[i], sizeof(float) * h->in_dim, x + a * ldx,
                                  sizeof(float) * ldx, sizeof(float) * h->in_dim, rows,
                                  cudaMemcpyHostToDevice, si);
    if (err != cudaSuccess) break;
    const FeatureArgs fa = feature_args(p, h->xd[i], rows, h->in_dim, h->in_dim, Cs, G);
    err = p->L > 15 ? launch_features_multipass(fa, h->pd[i], nullptr, nullptr, 0, nullptr, h->sc[i], si)
                    : launch_features(fa, h->pd[i], si);
    if (err != cudaSuccess) break;
    err = cudaMemcpyAsync(phi + a * F, h->pd[i], sizeof(float) * rows * F, cudaMemcpyDeviceToHost, si);
  }
  for (int i = 0; err == cudaSuccess && i < k; ++i) {
    err = cudaEventRecord(h->done[i], h->st[i]);
    if (err == cudaSuccess) err = cudaStreamWaitEvent(s, h->done[i], 0);
  }
  return launched(err, "mck_features_host");
}
