// tp_peaks.cu -- microbenchmarks of the hardware rates that bound the history
// loop: FP32 FMA, INT32 multiply-add and logic, the special-function unit
// (lg2, ex2, sin), FP64 FMA, FP64 global atomics (spread over the bins of a
// tally and piled on a few bins) and L2 read bandwidth.  The transport kernels
// are bound by instruction issue on these units, not by HBM and not by the
// tensor cores, so their roofline is taken against these measured rates.
//
// Every kernel runs a fixed number of iterations of independent dependency
// chains (enough chains per thread to hide the pipeline latency), keeps its
// result live by writing one value per thread, and is timed with CUDA events
// on the caller's stream after one warm-up launch.  Lane operations per second
// = threads x iterations x chains / time.
#include <cuda_runtime.h>

#include <algorithm>
#include <cstdint>

#include "tp_internal.h"

namespace {

constexpr int kChains = 8;     // independent chains per thread
constexpr int kBlock = 256;

__global__ void __launch_bounds__(kBlock) k_fma32(float* out, int iters, float b, float c) {
  float a[kChains];
#pragma unroll
  for (int i = 0; i < kChains; ++i) a[i] = (float)(threadIdx.x + i);
  for (int it = 0; it < iters; ++it) {
#pragma unroll
    for (int i = 0; i < kChains; ++i) a[i] = fmaf(a[i], b, c);
  }
  float s = 0.f;
#pragma unroll
  for (int i = 0; i < kChains; ++i) s += a[i];
  out[blockIdx.x * blockDim.x + threadIdx.x] = s;
}

// integer multiply-add (the Philox multiplies) and logic (its xors), in
// separate kernels since they run on different pipes
__global__ void __launch_bounds__(kBlock) k_imad(uint32_t* out, int iters, uint32_t m, uint32_t c) {
  uint32_t a[kChains];
#pragma unroll
  for (int i = 0; i < kChains; ++i) a[i] = threadIdx.x * 7u + i;
  for (int it = 0; it < iters; ++it) {
#pragma unroll
    for (int i = 0; i < kChains; ++i) a[i] = a[i] * m + c;
  }
  uint32_t s = 0;
#pragma unroll
  for (int i = 0; i < kChains; ++i) s ^= a[i];
  out[blockIdx.x * blockDim.x + threadIdx.x] = s;
}

__global__ void __launch_bounds__(kBlock) k_lop(uint32_t* out, int iters, uint32_t k0, uint32_t k1) {
  uint32_t a[kChains];
#pragma unroll
  for (int i = 0; i < kChains; ++i) a[i] = threadIdx.x * 13u + i;
  for (int it = 0; it < iters; ++it) {
#pragma unroll
    for (int i = 0; i < kChains; ++i) a[i] = (a[i] ^ k0) & (a[i] | k1);   // one three-input logic op
  }
  uint32_t s = 0;
#pragma unroll
  for (int i = 0; i < kChains; ++i) s += a[i];
  out[blockIdx.x * blockDim.x + threadIdx.x] = s;
}

template <int OP>
__device__ __forceinline__ float mufu(float x) {
  float y;
  if (OP == 0) asm volatile("lg2.approx.f32 %0, %1;" : "=f"(y) : "f"(x));
  else if (OP == 1) asm volatile("ex2.approx.f32 %0, %1;" : "=f"(y) : "f"(x));
  else asm volatile("sin.approx.f32 %0, %1;" : "=f"(y) : "f"(x));
  return y;
}

template <int OP>
__global__ void __launch_bounds__(kBlock) k_mufu(float* out, int iters) {
  float a[kChains];
#pragma unroll
  for (int i = 0; i < kChains; ++i) a[i] = 0.5f + 0.01f * (float)((threadIdx.x + i) & 31);
  for (int it = 0; it < iters; ++it) {
#pragma unroll
    for (int i = 0; i < kChains; ++i) a[i] = mufu<OP>(a[i]);
  }
  float s = 0.f;
#pragma unroll
  for (int i = 0; i < kChains; ++i) s += a[i];
  out[blockIdx.x * blockDim.x + threadIdx.x] = s;
}

__global__ void __launch_bounds__(kBlock) k_fma64(double* out, int iters, double b, double c) {
  double a[kChains];
#pragma unroll
  for (int i = 0; i < kChains; ++i) a[i] = (double)(threadIdx.x + i);
  for (int it = 0; it < iters; ++it) {
#pragma unroll
    for (int i = 0; i < kChains; ++i) a[i] = fma(a[i], b, c);
  }
  double s = 0.0;
#pragma unroll
  for (int i = 0; i < kChains; ++i) s += a[i];
  out[blockIdx.x * blockDim.x + threadIdx.x] = s;
}

// FP64 atomic adds into `nbins` bins (resident in L2): each thread walks the
// bins with a stride that spreads a warp's lanes over distinct bins.
__global__ void __launch_bounds__(kBlock) k_atomic64(double* bins, int nbins, int iters) {
  const unsigned t = blockIdx.x * blockDim.x + threadIdx.x;
  unsigned b = (t * 2654435761u) % (unsigned)nbins;
  for (int it = 0; it < iters; ++it) {
    atomicAdd(bins + b, 1.0);
    b = (b + 97u) % (unsigned)nbins;   // stays in [0, nbins) for any nbins
  }
}

// L2 read bandwidth: every block reads the whole (L2-resident) buffer in
// 16-byte loads, `passes` times.
__global__ void __launch_bounds__(kBlock) k_l2read(const float4* __restrict__ buf, size_t n4, int passes,
                                                   float* out) {
  float4 acc = make_float4(0.f, 0.f, 0.f, 0.f);
  const size_t stride = (size_t)gridDim.x * blockDim.x;
  for (int p = 0; p < passes; ++p) {
    for (size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x; i < n4; i += stride) {
      const float4 v = __ldcg(buf + i);
      acc.x += v.x; acc.y += v.y; acc.z += v.z; acc.w += v.w;
    }
  }
  out[blockIdx.x * blockDim.x + threadIdx.x] = acc.x + acc.y + acc.z + acc.w;
}

// SM clock during a launch: clock64 cycles over globaltimer nanoseconds.
__global__ void k_clock(unsigned long long* out, int iters, float b, float c) {
  unsigned long long c0 = clock64(), t0;
  asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t0));
  float a[kChains];
#pragma unroll
  for (int i = 0; i < kChains; ++i) a[i] = (float)(threadIdx.x + i);
  for (int it = 0; it < iters; ++it) {
#pragma unroll
    for (int i = 0; i < kChains; ++i) a[i] = fmaf(a[i], b, c);
  }
  unsigned long long c1 = clock64(), t1;
  asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t1));
  float s = 0.f;
#pragma unroll
  for (int i = 0; i < kChains; ++i) s += a[i];
  if (threadIdx.x == 0 && blockIdx.x == 0) {
    out[0] = c1 - c0;
    out[1] = t1 - t0;
    out[2] = (unsigned long long)(s != 12345.f);
  }
}

}  // namespace

extern "C" tp_status tp_measure_peaks(tp_peaks* out, void* stream) {
  if (!out) return TP_ERR_INVALID_ARG;
  cudaStream_t st = (cudaStream_t)stream;
  int dev = 0, sms = 0;
  if (cudaGetDevice(&dev) != cudaSuccess) return TP_ERR_CUDA;
  if (cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess) return TP_ERR_CUDA;
  const int grid = sms * 8;                       // 8 blocks of 256 threads per SM: full occupancy
  const size_t threads = (size_t)grid * kBlock;
  const int nbins = 3600;                         // the powder workload's detector
  const size_t l2_bytes = 32ull << 20;            // well inside L2
  void* scratch = nullptr;
  const size_t need = threads * sizeof(double) + nbins * sizeof(double) + l2_bytes + 64;
  if (cudaMalloc(&scratch, need) != cudaSuccess) return TP_ERR_OOM;
  uint8_t* base = static_cast<uint8_t*>(scratch);
  void* sink = base;
  double* bins = reinterpret_cast<double*>(base + threads * sizeof(double));
  float4* l2buf = reinterpret_cast<float4*>(base + threads * sizeof(double) + nbins * sizeof(double));
  unsigned long long* clk = reinterpret_cast<unsigned long long*>(reinterpret_cast<uint8_t*>(l2buf) + l2_bytes);
  cudaEvent_t a, b;
  cudaEventCreate(&a);
  cudaEventCreate(&b);
  cudaError_t err = cudaMemsetAsync(scratch, 0, need, st);
  // times launch() (after one warm-up launch); returns seconds
  auto timed = [&](auto launch) -> double {
    launch();
    cudaEventRecord(a, st);
    launch();
    cudaEventRecord(b, st);
    if (cudaEventSynchronize(b) != cudaSuccess) return -1.0;
    float ms = 0.f;
    cudaEventElapsedTime(&ms, a, b);
    return ms * 1e-3;
  };
  const int it32 = 4096, itmufu = 1024, it64 = 32, itat = 256;
  const double lanes = (double)threads * kChains;
  double t;
  t = timed([&] { k_fma32<<<grid, kBlock, 0, st>>>((float*)sink, it32, 0.999f, 0.001f); });
  out->fp32_fma = lanes * it32 / t;
  t = timed([&] { k_imad<<<grid, kBlock, 0, st>>>((uint32_t*)sink, it32, 0xD2511F53u, 0x9E3779B9u); });
  out->int32_imad = lanes * it32 / t;
  t = timed([&] { k_lop<<<grid, kBlock, 0, st>>>((uint32_t*)sink, it32, 0x9E3779B9u, 0xBB67AE85u); });
  out->int32_logic = lanes * it32 / t;
  t = timed([&] { k_mufu<0><<<grid, kBlock, 0, st>>>((float*)sink, itmufu); });
  out->mufu_lg2 = lanes * itmufu / t;
  t = timed([&] { k_mufu<1><<<grid, kBlock, 0, st>>>((float*)sink, itmufu); });
  out->mufu_ex2 = lanes * itmufu / t;
  t = timed([&] { k_mufu<2><<<grid, kBlock, 0, st>>>((float*)sink, itmufu); });
  out->mufu_sin = lanes * itmufu / t;
  t = timed([&] { k_fma64<<<grid, kBlock, 0, st>>>((double*)sink, it64, 0.999, 0.001); });
  out->fp64_fma = lanes * it64 / t;
  t = timed([&] { k_atomic64<<<grid, kBlock, 0, st>>>(bins, nbins, itat); });
  out->atomic_f64_spread = (double)threads * itat / t;
  t = timed([&] { k_atomic64<<<grid, kBlock, 0, st>>>(bins, 32, itat); });
  out->atomic_f64_hot = (double)threads * itat / t;
  const int passes = 8;
  t = timed([&] { k_l2read<<<grid, kBlock, 0, st>>>(l2buf, l2_bytes / 16, passes, (float*)sink); });
  out->l2_read_bytes = (double)l2_bytes * passes / t;
  t = timed([&] { k_clock<<<sms, kBlock, 0, st>>>(clk, it32, 0.999f, 0.001f); });
  unsigned long long h[3] = {0, 0, 0};
  if (cudaMemcpyAsync(h, clk, sizeof h, cudaMemcpyDeviceToHost, st) == cudaSuccess) cudaStreamSynchronize(st);
  out->sm_clock_mhz = h[1] > 0 ? 1e3 * (double)h[0] / (double)h[1] : 0.0;
  out->sm_count = sms;
  if (err == cudaSuccess) err = cudaGetLastError();
  cudaEventDestroy(a);
  cudaEventDestroy(b);
  cudaFree(scratch);
  return err == cudaSuccess ? TP_OK : TP_ERR_CUDA;
}
