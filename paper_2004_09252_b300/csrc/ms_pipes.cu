// Integer pipe probe: sustained lane operations per SM per clock of the
// 32-bit op classes the cipher is made of (add, xor, funnel shift, byte
// permute, multiply-add, multiply-high) and of mixes of them.  This is the
// measurement behind the kernel rooflines, not part of the method.
//
// The grid is 4 CTAs of 256 threads per SM; each thread advances 8
// independent dependency chains for kIters iterations, so the issue slots,
// not the latency, limit the rate.  The rate is the kernel's CUDA-event time
// over all SMs; the SM clock comes from clock64 against %globaltimer.
#include <cstring>
#include <vector>

#include "ms_internal.h"

namespace {

constexpr int kIters = 16384;
constexpr int kChains = 8;
constexpr int kCtasPerSm = 4;
constexpr int kThreads = 256;

__device__ __forceinline__ unsigned long long gtime() {
  unsigned long long t;
  asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
  return t;
}

__device__ __forceinline__ void op_add(uint32_t &x, uint32_t y) { asm volatile("add.u32 %0, %0, %1;" : "+r"(x) : "r"(y)); }
__device__ __forceinline__ void op_xor(uint32_t &x, uint32_t y) { asm volatile("xor.b32 %0, %0, %1;" : "+r"(x) : "r"(y)); }
__device__ __forceinline__ void op_shf(uint32_t &x) { asm volatile("shf.l.wrap.b32 %0, %0, %0, 7;" : "+r"(x)); }
__device__ __forceinline__ void op_prmt(uint32_t &x, uint32_t y) {
  asm volatile("prmt.b32 %0, %0, %1, 0x1032;" : "+r"(x) : "r"(y));
}
__device__ __forceinline__ void op_mad(uint32_t &x, uint32_t m, uint32_t y) {
  asm volatile("mad.lo.u32 %0, %0, %1, %2;" : "+r"(x) : "r"(m), "r"(y));
}
__device__ __forceinline__ void op_mulhi(uint32_t &x, uint32_t m) { asm volatile("mul.hi.u32 %0, %0, %1;" : "+r"(x) : "r"(m)); }

template <int OP>
__global__ void __launch_bounds__(kThreads) k_pipe(uint32_t *out, uint32_t seed, uint32_t m,
                                                   unsigned long long *clk) {
  uint32_t x[kChains];
  const uint32_t y = seed ^ threadIdx.x;
#pragma unroll
  for (int i = 0; i < kChains; ++i) x[i] = seed * (i + 1) + threadIdx.x + blockIdx.x;
  const unsigned long long c0 = clock64(), g0 = gtime();
#pragma unroll 1
  for (int it = 0; it < kIters; ++it) {
#pragma unroll
    for (int i = 0; i < kChains; ++i) {
      switch (OP) {
        case MS_PIPE_ADD: op_add(x[i], y); break;
        case MS_PIPE_XOR: op_xor(x[i], y); break;
        case MS_PIPE_SHF: op_shf(x[i]); break;
        case MS_PIPE_PRMT: op_prmt(x[i], y); break;
        case MS_PIPE_MAD: op_mad(x[i], m, y); break;
        case MS_PIPE_MULHI: op_mulhi(x[i], m); break;
        case MS_PIPE_XOR_MAD: if (i & 1) op_mad(x[i], m, y); else op_xor(x[i], y); break;
        case MS_PIPE_SHF_MAD: if (i & 1) op_mad(x[i], m, y); else op_shf(x[i]); break;
        case MS_PIPE_XOR_ADD: if (i & 1) op_add(x[i], y); else op_xor(x[i], y); break;
        case MS_PIPE_XOR_SHF: if (i & 1) op_shf(x[i]); else op_xor(x[i], y); break;
        default: break;
      }
    }
  }
  const unsigned long long c1 = clock64(), g1 = gtime();
  uint32_t acc = 0;
#pragma unroll
  for (int i = 0; i < kChains; ++i) acc ^= x[i];
  out[blockIdx.x * blockDim.x + threadIdx.x] = acc;  // keeps the chains live
  if (threadIdx.x == 0) {
    clk[2 * blockIdx.x] = c1 - c0;
    clk[2 * blockIdx.x + 1] = g1 - g0;
  }
}

using PipeFn = void (*)(uint32_t *, uint32_t, uint32_t, unsigned long long *);

const PipeFn kFns[MS_PIPE_CLASSES] = {
    &k_pipe<MS_PIPE_ADD>,     &k_pipe<MS_PIPE_XOR>,     &k_pipe<MS_PIPE_SHF>,     &k_pipe<MS_PIPE_PRMT>,
    &k_pipe<MS_PIPE_MAD>,     &k_pipe<MS_PIPE_MULHI>,   &k_pipe<MS_PIPE_XOR_MAD>, &k_pipe<MS_PIPE_SHF_MAD>,
    &k_pipe<MS_PIPE_XOR_ADD>, &k_pipe<MS_PIPE_XOR_SHF>,
};

}  // namespace

extern "C" int ms_probe_int_pipes(int device, ms_pipe_rate *out, size_t n_out) {
  if (!out || n_out < MS_PIPE_CLASSES) return MS_EINVAL;
  int ndev = 0;
  if (cudaGetDeviceCount(&ndev) != cudaSuccess || device < 0 || device >= ndev) {
    cudaGetLastError();
    return MS_EINVAL;
  }
  ms::DeviceGuard g(device);
  int sms = 0;
  if (cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, device) != cudaSuccess || sms < 1) {
    cudaGetLastError();
    return MS_ECUDA;
  }
  const int grid = sms * kCtasPerSm;
  uint32_t *d_out = nullptr;
  unsigned long long *d_clk = nullptr;
  cudaStream_t s = nullptr;
  cudaEvent_t a = nullptr, b = nullptr;
  cudaError_t e = cudaMalloc(&d_out, (size_t)grid * kThreads * sizeof(uint32_t));
  if (e == cudaSuccess) e = cudaMalloc(&d_clk, 2 * (size_t)grid * sizeof(unsigned long long));
  if (e == cudaSuccess) e = cudaStreamCreateWithFlags(&s, cudaStreamNonBlocking);
  if (e == cudaSuccess) e = cudaEventCreate(&a);
  if (e == cudaSuccess) e = cudaEventCreate(&b);
  std::vector<unsigned long long> h(2 * (size_t)grid);
  for (int op = 0; op < MS_PIPE_CLASSES && e == cudaSuccess; ++op) {
    kFns[op]<<<grid, kThreads, 0, s>>>(d_out, 12345u, 4096u, d_clk);  // warm-up
    e = cudaGetLastError();
    if (e == cudaSuccess) e = cudaEventRecord(a, s);
    if (e == cudaSuccess) {
      kFns[op]<<<grid, kThreads, 0, s>>>(d_out, 12345u, 4096u, d_clk);
      e = cudaGetLastError();
    }
    if (e == cudaSuccess) e = cudaEventRecord(b, s);
    if (e == cudaSuccess) e = cudaEventSynchronize(b);
    float ms = 0;
    if (e == cudaSuccess) e = cudaEventElapsedTime(&ms, a, b);
    if (e == cudaSuccess) e = cudaMemcpy(h.data(), d_clk, h.size() * sizeof(unsigned long long), cudaMemcpyDeviceToHost);
    if (e != cudaSuccess) break;
    double cyc = 0, ns = 0;
    for (int i = 0; i < grid; ++i) {
      cyc += (double)h[2 * i];
      ns += (double)h[2 * i + 1];
    }
    cyc /= grid;
    ns /= grid;
    const double lane_ops = (double)kIters * kChains * kThreads * grid;
    ms_pipe_rate &r = out[op];
    std::memset(&r, 0, sizeof(r));
    r.op_class = op;
    r.sm_mhz = ns > 0 ? cyc / ns * 1e3 : 0.0;
    r.tops = ms > 0 ? lane_ops / (ms * 1e-3) / 1e12 : 0.0;
    // whole-GPU rate per SM per clock: the kernel's event time, the measured
    // clock (per-CTA intervals would assume every SM holds the same CTAs
    // for the whole run, which the block scheduler does not promise)
    r.lanes_per_sm_clk = r.sm_mhz > 0 ? r.tops * 1e12 / sms / (r.sm_mhz * 1e6) : 0.0;
  }
  if (a) cudaEventDestroy(a);
  if (b) cudaEventDestroy(b);
  if (s) cudaStreamDestroy(s);
  if (d_out) cudaFree(d_out);
  if (d_clk) cudaFree(d_clk);
  if (e != cudaSuccess) {
    cudaGetLastError();
    return e == cudaErrorMemoryAllocation ? MS_ENOMEM : MS_ECUDA;
  }
  return MS_OK;
}
