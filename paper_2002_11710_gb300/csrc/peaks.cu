// peaks.cu - microbenchmarks of one SM's integer issue rate and shared-memory load rate:
// the measured denominators of the roofline of the Tabu kernels, whose hot loop is
// int32 add / compare / min / select on values gathered from shared memory (no tensor
// cores apply, and HBM is touched only once per launch).
//
// Each probe fills every SM with resident CTAs; each CTA records its SM id and the SM
// clock (clock64) after a block barrier at the start and at the end of a fixed amount
// of work, so the host gets, per SM, (work of its CTAs) / (cycles from the first start to
// the last end). Work is counted in the units the roofline uses:
//   ASCHED_PROBE_INT32        int32 operations (add, xor, min; 8 independent chains per
//                             thread, so issue and not latency bounds it);
//   ASCHED_PROBE_INT32_ADD_XOR the same without the min;
//   ASCHED_PROBE_LDS          32-bit shared-memory words loaded, conflict-free (the 32
//                             lanes of a warp read 32 distinct banks);
//   ASCHED_PROBE_LDS_GATHER   the same with every lane at a random word of a 64 KB table
//                             (the bank conflicts of random gathers included).
#include <cuda_runtime.h>
#include <stdint.h>

#include "asched.h"

namespace {

constexpr int kChains = 8;
constexpr int kUnroll = 4;
constexpr int kTabWords = 16384;  // 64 KB table for the load probes
constexpr int kLoadsPerStep = ASCHED_PROBE_LDS_LOADS_PER_STEP;
static_assert(kChains * kUnroll * 3 == ASCHED_PROBE_INT32_OPS_PER_STEP, "ops per step");
static_assert(kChains * kUnroll * 2 == ASCHED_PROBE_INT32_ADD_XOR_OPS_PER_STEP, "ops per step");
static_assert(kTabWords / 2 + 32 * kLoadsPerStep <= kTabWords, "loads stay inside the table");

__device__ __forceinline__ uint32_t sm_id() {
  uint32_t r;
  asm volatile("mov.u32 %0, %%smid;" : "=r"(r));
  return r;
}

__device__ __forceinline__ void record(int64_t* rec, long long t0, long long t1) {
  if (threadIdx.x == 0) {
    rec[3 * blockIdx.x + 0] = sm_id();
    rec[3 * blockIdx.x + 1] = t0;
    rec[3 * blockIdx.x + 2] = t1;
  }
}

// MIN: add / xor / min per chain and step; otherwise add / xor (no reassociation can
// merge the steps of a chain: every add is followed by an xor).
template <bool MIN>
__global__ void probe_int32_kernel(int iters, uint32_t c, uint32_t d, uint32_t e, int64_t* rec, uint32_t* sink) {
  uint32_t a[kChains];
#pragma unroll
  for (int k = 0; k < kChains; ++k) a[k] = threadIdx.x * (k + 3) + blockIdx.x;
  __syncthreads();
  const long long t0 = clock64();
  for (int i = 0; i < iters; ++i) {
#pragma unroll
    for (int u = 0; u < kUnroll; ++u) {
#pragma unroll
      for (int k = 0; k < kChains; ++k) {
        asm("add.u32 %0, %0, %1;" : "+r"(a[k]) : "r"(c));
        asm("xor.b32 %0, %0, %1;" : "+r"(a[k]) : "r"(d));
        if (MIN) asm("min.u32 %0, %0, %1;" : "+r"(a[k]) : "r"(e));
      }
    }
  }
  __syncthreads();
  const long long t1 = clock64();
  record(rec, t0, t1);
  uint32_t x = 0;
#pragma unroll
  for (int k = 0; k < kChains; ++k) x ^= a[k];
  if (x == 0x9E3779B9u) sink[blockIdx.x] = x;  // keeps the chains live; practically never stored
}

template <bool GATHER>
__global__ void probe_lds_kernel(int iters, int64_t* rec, uint32_t* sink) {
  extern __shared__ uint32_t tab[];
  for (int i = threadIdx.x; i < kTabWords; i += blockDim.x) tab[i] = i * 2654435761u;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  // conflict-free: lane l reads bank l; gather: every lane starts at its own random word
  uint32_t h = (blockIdx.x * 1024u + threadIdx.x) * 2654435761u;
  uint32_t base = GATHER ? (h >> 18) : static_cast<uint32_t>(warp * 32 * kLoadsPerStep + lane);
  uint32_t acc = 0;
  __syncthreads();
  const long long t0 = clock64();
  for (int i = 0; i < iters; ++i) {
    // a start in the table's first half: the step's loads (up to 32 * 15 words further)
    // stay inside the table
    const uint32_t b = base & (kTabWords / 2 - 1) & ~(GATHER ? 0u : 31u);
    const uint32_t* p = tab + (GATHER ? b : (b | lane));
#pragma unroll
    for (int k = 0; k < kLoadsPerStep; ++k) acc += p[k * 32];
    if (GATHER) {
      h = h * 1664525u + 1013904223u;  // next random start (linear congruential step)
      base = h >> 18;
    } else {
      base += 32 * kLoadsPerStep;
    }
  }
  __syncthreads();
  const long long t1 = clock64();
  record(rec, t0, t1);
  if (acc == 0x9E3779B9u) sink[blockIdx.x] = acc;
}

int launch_probe(void* fn, int threads, size_t smem, void** args, int64_t* rec, int rec_ctas, int32_t* ctas_out,
                 cudaStream_t st) {
  int dev = 0, sms = 0, per_sm = 0;
  if (smem > 48 * 1024 && cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                                static_cast<int>(smem)) != cudaSuccess)
    return ASCHED_E_CUDA;
  if (cudaGetDevice(&dev) != cudaSuccess ||
      cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess ||
      cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, fn, threads, smem) != cudaSuccess) {
    (void)cudaGetLastError();
    return ASCHED_E_CUDA;
  }
  const int ctas = sms * per_sm;
  if (per_sm < 1) return ASCHED_E_TOO_LARGE;
  if (ctas > rec_ctas) return ASCHED_E_INVALID;
  if (cudaLaunchKernel(fn, dim3(ctas), dim3(threads), args, smem, st) != cudaSuccess) {
    (void)cudaGetLastError();
    return ASCHED_E_CUDA;
  }
  *ctas_out = ctas;
  return ASCHED_OK;
}

}  // namespace

extern "C" int asched_probe_sm_peak(int32_t kind, int32_t iters, int64_t* rec, int32_t rec_ctas, uint32_t* sink,
                                    int32_t* ctas_out, int32_t* threads_out, void* stream) {
  if (!rec || !sink || !ctas_out || !threads_out || iters < 1 || rec_ctas < 1) return ASCHED_E_INVALID;
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  const int threads = 512;
  *threads_out = threads;
  if (kind == ASCHED_PROBE_INT32 || kind == ASCHED_PROBE_INT32_ADD_XOR) {
    uint32_t c = 0x9E37u, d = 0x5bd1e995u, e = 0xFFFFFF00u;
    void* args[] = {&iters, &c, &d, &e, &rec, &sink};
    void* fn = kind == ASCHED_PROBE_INT32 ? reinterpret_cast<void*>(&probe_int32_kernel<true>)
                                          : reinterpret_cast<void*>(&probe_int32_kernel<false>);
    return launch_probe(fn, threads, 0, args, rec, rec_ctas, ctas_out, st);
  }
  if (kind == ASCHED_PROBE_LDS || kind == ASCHED_PROBE_LDS_GATHER) {
    void* args[] = {&iters, &rec, &sink};
    void* fn = kind == ASCHED_PROBE_LDS ? reinterpret_cast<void*>(&probe_lds_kernel<false>)
                                        : reinterpret_cast<void*>(&probe_lds_kernel<true>);
    return launch_probe(fn, threads, kTabWords * 4, args, rec, rec_ctas, ctas_out, st);
  }
  return ASCHED_E_INVALID;
}
