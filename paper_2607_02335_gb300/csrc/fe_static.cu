// fe_static.cu -- duality pairing without any device allocation (fe_pairing_noalloc).
//
// Some callers cannot let the library call cudaMalloc: a host process that has handed the whole
// device memory to its own pool (a caching allocator, or a serving loop that admits work against
// a fixed memory budget), or a latency-critical loop where an allocation (which may synchronize
// the device) is not acceptable.  fe_pairing keeps its per-CTA partial sums in a buffer the mesh
// allocates on first use; this variant keeps them in a file-scope static device array instead, so
// every call allocates nothing.
//
// Scratch: FE_PAIRING_NOALLOC_MAX_PARTIALS doubles (64 KiB) on every device that loads the
// library, held until the process exits.  One CTA reduces FE_PAIRING_NOALLOC_CHUNK consecutive
// entries into one partial, so vectors are limited to MAX_PARTIALS * CHUNK entries; longer ones are
// rejected with FE_ERR_INVALID.  Every call shares the array and overwrites the partials it reads
// (each CTA writes its slot before the finishing kernel reads it), so nothing has to be cleared;
// calls that overlap on the GPU (different streams, no ordering) race on the array.
// The host needs the array's device address: in host code the symbol names a host-side stand-in,
// so the first call on each device looks it up with cudaGetSymbolAddress while that device is
// current; that first call should therefore come before any stream capture.
#include <mutex>

#include "fe_vec.cuh"

#define FE_PAIRING_NOALLOC_MAX_PARTIALS 8192
#define FE_PAIRING_NOALLOC_CHUNK (RED_THREADS * 32)
#define FE_MAX_DEVICES 64

static __device__ __align__(256) double g_pairing_partials[FE_PAIRING_NOALLOC_MAX_PARTIALS];

// one partial per CTA over its chunk [blockIdx.x * CHUNK, min(n, (blockIdx.x + 1) * CHUNK)),
// binary64 products and sums as in fe_pairing
template <class S>
__global__ void __launch_bounds__(RED_THREADS)
    k_pairing_chunk(const S* __restrict__ a, const S* __restrict__ b, long long n,
                    double* __restrict__ partials) {
  __shared__ double sh[32];
  const long long lo = (long long)blockIdx.x * FE_PAIRING_NOALLOC_CHUNK;
  long long hi = lo + FE_PAIRING_NOALLOC_CHUNK;
  if (hi > n) hi = n;
  double acc = 0.0;
  for (long long e = lo + threadIdx.x; e < hi; e += RED_THREADS)
    acc = fma((double)__ldg(a + e), (double)__ldg(b + e), acc);
  acc = block_reduce_f64(acc, sh);
  if (threadIdx.x == 0) partials[blockIdx.x] = acc;
}

// sum of the first nparts partials in a fixed order
__global__ void __launch_bounds__(RED_THREADS)
    k_pairing_chunk_sum(const double* __restrict__ partials, int nparts, double* __restrict__ out) {
  __shared__ double sh[32];
  double acc = 0.0;
  for (int i = threadIdx.x; i < nparts; i += RED_THREADS) acc += partials[i];
  acc = block_reduce_f64(acc, sh);
  if (threadIdx.x == 0) out[0] = acc;
}

// device address of the static array, looked up once per device with that device current
static fe_status scratch_for_device(int dev, double** out) {
  static std::mutex mu;
  static double* addr[FE_MAX_DEVICES] = {};
  if (dev < 0 || dev >= FE_MAX_DEVICES) {
    fe_set_error("fe_pairing_noalloc: device ordinal %d out of range", dev);
    return FE_ERR_INVALID;
  }
  std::lock_guard<std::mutex> lock(mu);
  if (!addr[dev]) {
    void* p = nullptr;
    FE_CUDA(cudaGetSymbolAddress(&p, g_pairing_partials), "fe_pairing_noalloc: cudaGetSymbolAddress");
    addr[dev] = static_cast<double*>(p);
  }
  *out = addr[dev];
  return FE_OK;
}

extern "C" fe_status fe_pairing_noalloc(const fe_mesh* m, fe_prec prec, const void* a,
                                        const void* b, double* result_dev, void* stream) {
  if (!m || !a || !b || !result_dev) {
    fe_set_error("fe_pairing_noalloc: null argument");
    return FE_ERR_INVALID;
  }
  if (!fe_aligned(a) || !fe_aligned(b)) {
    fe_set_error("fe_pairing_noalloc: vectors must be 16-byte aligned");
    return FE_ERR_INVALID;
  }
  if (prec != FE_F64 && prec != FE_F32) {
    fe_set_error("fe_pairing_noalloc: precision %d not provided", (int)prec);
    return FE_ERR_INVALID;
  }
  const long long n = m->ncw;
  const long long nparts = (n + FE_PAIRING_NOALLOC_CHUNK - 1) / FE_PAIRING_NOALLOC_CHUNK;
  if (nparts > FE_PAIRING_NOALLOC_MAX_PARTIALS) {
    fe_set_error("fe_pairing_noalloc: %lld cell-wise entries exceed the static scratch limit of %lld "
                 "entries; use fe_pairing",
                 n, (long long)FE_PAIRING_NOALLOC_MAX_PARTIALS * FE_PAIRING_NOALLOC_CHUNK);
    return FE_ERR_INVALID;
  }
  FeDeviceGuard device_guard;
  FE_CUDA(device_guard.set(m->d.device), "cudaSetDevice");
  double* scratch = nullptr;
  FE_TRY(scratch_for_device(m->d.device, &scratch));
  cudaStream_t st = (cudaStream_t)stream;
  if (nparts > 0) {
    if (prec == FE_F64)
      k_pairing_chunk<double><<<(unsigned)nparts, RED_THREADS, 0, st>>>(
          (const double*)a, (const double*)b, n, scratch);
    else
      k_pairing_chunk<float><<<(unsigned)nparts, RED_THREADS, 0, st>>>(
          (const float*)a, (const float*)b, n, scratch);
  }
  k_pairing_chunk_sum<<<1, RED_THREADS, 0, st>>>(scratch, (int)nparts, result_dev);
  return fe_cuda_check(cudaGetLastError(), "fe_pairing_noalloc launch");
}
