// Throughput probe of the integer pipes the classification runs on: how many
// LOP3, PRMT, SHF and IMAD operations an SM retires per clock, alone and with
// PRMT and IMAD mixed.  It measures the denominator of the integer-ALU
// roofline (the classification's ops per byte times bytes per second against
// SMs x ops per clock x clock); it is not part of the validator.
//
// Every thread runs kChains independent dependency chains of one operation,
// so that issue, not latency, limits the rate; a full grid (2048 threads per
// SM) runs `iters` rounds.  The launch is timed with CUDA events: operations
// per second, divided by SMs and the SM clock the caller sampled, give
// operations per clock per SM.  (Each block also records the span of its
// loop in clock64() ticks.)
#include <cuda_runtime.h>
#include <stdint.h>

namespace {

constexpr int kChains = 8;
constexpr int kThreads = 256;

template <int OP>
__device__ __forceinline__ uint32_t step(uint32_t a, uint32_t b) {
  uint32_t d;
  if constexpr (OP == 0) {  // LOP3 (three-input xor)
    asm volatile("lop3.b32 %0, %1, %2, %3, 0x96;" : "=r"(d) : "r"(a), "r"(b), "r"(0x5A5A5A5Au));
  } else if constexpr (OP == 1) {  // PRMT: a table lookup indexed by the chain value
    asm volatile("prmt.b32 %0, %1, %2, %3;" : "=r"(d) : "r"(b), "r"(0x13579BDFu), "r"(a));
  } else if constexpr (OP == 2) {  // SHF: funnel shift
    asm volatile("shf.l.wrap.b32 %0, %1, %2, 5;" : "=r"(d) : "r"(a), "r"(b));
  } else {  // IMAD
    asm volatile("mad.lo.u32 %0, %1, %2, %3;" : "=r"(d) : "r"(a), "r"(0x01000193u), "r"(b));
  }
  return d;
}

// OP 0..3: one operation; OP 4: PRMT and IMAD chains interleaved 1:1.
template <int OP>
__global__ void __launch_bounds__(kThreads) probe_kernel(uint32_t iters, uint32_t seed,
                                                          uint32_t* sink, long long* cycles) {
  uint32_t a[kChains];
  const uint32_t b = seed ^ threadIdx.x;
#pragma unroll
  for (int k = 0; k < kChains; ++k) a[k] = seed * (k + 1) + threadIdx.x;
  __syncthreads();
  const long long t0 = clock64();
  for (uint32_t i = 0; i < iters; ++i) {
#pragma unroll
    for (int k = 0; k < kChains; ++k) {
      if constexpr (OP == 4) a[k] = (k & 1) ? step<3>(a[k], b) : step<1>(a[k], b);
      else a[k] = step<OP>(a[k], b);
    }
  }
  __syncthreads();
  const long long t1 = clock64();
  uint32_t x = 0;
#pragma unroll
  for (int k = 0; k < kChains; ++k) x ^= a[k];
  if (x == 0x9E3779B9u) sink[0] = x;  // keeps the chains live
  if (threadIdx.x == 0) cycles[blockIdx.x] = t1 - t0;
}

template <int OP>
cudaError_t run(unsigned blocks, uint32_t iters, long long* cycles, uint32_t* sink) {
  probe_kernel<OP><<<blocks, kThreads>>>(iters, 0x2545F491u, sink, cycles);
  return cudaGetLastError();
}

}  // namespace

// op: 0 LOP3, 1 PRMT, 2 SHF, 3 IMAD, 4 PRMT+IMAD mixed.  cycles_out: host
// int64[blocks_per_sm * sm_count]; *ops_per_block receives the operations one
// block executes, *ms_out the launch's event time.  Returns 0 on success,
// else the CUDA error code.
extern "C" int alu_probe_run(int op, int blocks_per_sm, unsigned iters, long long* cycles_out,
                             double* ops_per_block, int* sm_count_out, float* ms_out) {
  int dev = 0, sms = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e == cudaSuccess) e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  if (e != cudaSuccess) return (int)e;
  const unsigned blocks = (unsigned)(sms * blocks_per_sm);
  long long* cyc = nullptr;
  uint32_t* sink = nullptr;
  cudaEvent_t t0 = nullptr, t1 = nullptr;
  e = cudaMalloc(&cyc, sizeof(long long) * blocks);
  if (e == cudaSuccess) e = cudaMalloc(&sink, sizeof(uint32_t));
  if (e == cudaSuccess) e = cudaEventCreate(&t0);
  if (e == cudaSuccess) e = cudaEventCreate(&t1);
  if (e == cudaSuccess) e = cudaEventRecord(t0);
  if (e == cudaSuccess) {
    switch (op) {
      case 0: e = run<0>(blocks, iters, cyc, sink); break;
      case 1: e = run<1>(blocks, iters, cyc, sink); break;
      case 2: e = run<2>(blocks, iters, cyc, sink); break;
      case 3: e = run<3>(blocks, iters, cyc, sink); break;
      default: e = run<4>(blocks, iters, cyc, sink); break;
    }
  }
  if (e == cudaSuccess) e = cudaEventRecord(t1);
  if (e == cudaSuccess) e = cudaDeviceSynchronize();
  if (e == cudaSuccess) e = cudaEventElapsedTime(ms_out, t0, t1);
  if (e == cudaSuccess)
    e = cudaMemcpy(cycles_out, cyc, sizeof(long long) * blocks, cudaMemcpyDeviceToHost);
  if (t0) cudaEventDestroy(t0);
  if (t1) cudaEventDestroy(t1);
  cudaFree(cyc);
  cudaFree(sink);
  *ops_per_block = (double)kThreads * kChains * (double)iters;
  *sm_count_out = sms;
  return (int)e;
}
