// vc_peaks.cu -- the measured denominators of the keystream's roofline: the
// binary64 pipe's throughput (independent fused multiply-adds), the 32-bit
// integer multiply-add throughput, and the dependency-chain latency of one
// PLCM step (Eq. 5) on the integer pipes, each timed on the device the call
// runs on.  None of these kernels touches the cipher's data.
#include <cuda_runtime.h>

#include <cstdint>

#include "vc_ieee.cuh"
#include "vcrypt.h"
#include "vcrypt_debug.h"

namespace {

constexpr int kPeakThreads = 256;
constexpr int kPeakChains = 8;   // independent chains per thread (hide the pipes' latency)
constexpr int kPeakIters = 2048;

// kPeakChains independent binary64 FMA chains per thread; the sum is written
// only if it equals the impossible sentinel, so nothing is optimised away.
__global__ void __launch_bounds__(kPeakThreads) k_peak_fp64(double b, double c, double* sink) {
  double a[kPeakChains];
#pragma unroll
  for (int k = 0; k < kPeakChains; k++) a[k] = (double)(threadIdx.x + k) * 1e-3;
  for (int i = 0; i < kPeakIters; i++) {
#pragma unroll
    for (int k = 0; k < kPeakChains; k++) a[k] = __fma_rn(a[k], b, c);
  }
  double s = 0;
#pragma unroll
  for (int k = 0; k < kPeakChains; k++) s += a[k];
  if (s == -12345.678) sink[blockIdx.x] = s;
}

// The same with 32-bit integer multiply-adds.
__global__ void __launch_bounds__(kPeakThreads) k_peak_imad(uint32_t b, uint32_t c, uint32_t* sink) {
  uint32_t a[kPeakChains];
#pragma unroll
  for (int k = 0; k < kPeakChains; k++) a[k] = threadIdx.x * 7u + k;
  for (int i = 0; i < kPeakIters; i++) {
#pragma unroll
    for (int k = 0; k < kPeakChains; k++) a[k] = a[k] * b + c;
  }
  uint32_t s = 0;
#pragma unroll
  for (int k = 0; k < kPeakChains; k++) s ^= a[k];
  if (s == 0x9E3779B9u && b == 0u) sink[blockIdx.x] = s;
}

// One lane runs `iters` dependent PLCM steps (the integer-pipe form) and
// reports the clock64 cycles per step; the other lanes of the warp idle.
__global__ void k_plcm_chain_latency(double x0, double p, int iters, long long* cycles, double* sink) {
  if (threadIdx.x != 0) return;
  vc::PlcmFx F;
  vc::make_plcm_fx(p, 0.5 - p, F);
  uint64_t xb = vc::ieee_bits(x0);
  bool ok = true;
  const long long t0 = clock64();
  // four steps per loop pass, as the keystream kernel runs them: the next
  // step's exponent is then read from the previous step's result directly
  for (int i = 0; i < iters; i += 4) {
    bool o0 = true, o1 = true, o2 = true, o3 = true;
    xb = vc::plcm_fx_step(xb, F, o0);
    xb = vc::plcm_fx_step(xb, F, o1);
    xb = vc::plcm_fx_step(xb, F, o2);
    xb = vc::plcm_fx_step(xb, F, o3);
    ok &= o0 & o1 & o2 & o3;
  }
  const long long t1 = clock64();
  cycles[0] = t1 - t0;
  sink[0] = ok ? vc::ieee_double(xb) : -1.0;
}

int time_kernel(void (*launch)(cudaStream_t), cudaStream_t st, float* ms) {
  cudaEvent_t a = nullptr, b = nullptr;
  if (cudaEventCreate(&a) != cudaSuccess || cudaEventCreate(&b) != cudaSuccess) return VC_ERR_CUDA;
  launch(st);  // warm-up
  cudaEventRecord(a, st);
  launch(st);
  cudaEventRecord(b, st);
  cudaError_t e = cudaEventSynchronize(b);
  if (e == cudaSuccess) e = cudaEventElapsedTime(ms, a, b);
  if (e == cudaSuccess) e = cudaGetLastError();
  cudaEventDestroy(a);
  cudaEventDestroy(b);
  return e == cudaSuccess ? VC_OK : VC_ERR_CUDA;
}

int g_blocks = 0;
void* g_sink = nullptr;

void launch_fp64(cudaStream_t st) {
  k_peak_fp64<<<g_blocks, kPeakThreads, 0, st>>>(0.999999, 1e-7, static_cast<double*>(g_sink));
}
void launch_imad(cudaStream_t st) {
  k_peak_imad<<<g_blocks, kPeakThreads, 0, st>>>(0x01000193u, 0x811C9DC5u, static_cast<uint32_t*>(g_sink));
}

int peak(void (*launch)(cudaStream_t), void* stream, double* ops_per_s) {
  if (!ops_per_s) return VC_ERR_ARG;
  int dev = 0, sms = 0;
  if (cudaGetDevice(&dev) != cudaSuccess ||
      cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess)
    return VC_ERR_CUDA;
  g_blocks = sms * 8;  // 64 warps per SM: every scheduler has independent work each cycle
  if (cudaMalloc(&g_sink, sizeof(double) * g_blocks) != cudaSuccess) {
    cudaGetLastError();
    return VC_ERR_OOM;
  }
  float ms = 0.f;
  const int rc = time_kernel(launch, (cudaStream_t)stream, &ms);
  cudaFree(g_sink);
  g_sink = nullptr;
  if (rc) return rc;
  const double ops = (double)g_blocks * kPeakThreads * kPeakIters * kPeakChains;
  *ops_per_s = ms > 0.f ? ops / (ms * 1e-3) : 0.0;
  return VC_OK;
}

}  // namespace

extern "C" int vc_dbg_fp64_peak(double* ops_per_s, void* stream) { return peak(launch_fp64, stream, ops_per_s); }

extern "C" int vc_dbg_imad_peak(double* ops_per_s, void* stream) { return peak(launch_imad, stream, ops_per_s); }

extern "C" int vc_dbg_plcm_latency(double x0, double p, int32_t iters, double* cycles_per_step, void* stream) {
  if (!cycles_per_step || iters < 1 || !(x0 > 0.0 && x0 < 1.0) || !(p > 0.0 && p < 0.5)) return VC_ERR_ARG;
  long long* d_cyc = nullptr;
  double* d_sink = nullptr;
  if (cudaMalloc(&d_cyc, sizeof(long long)) != cudaSuccess || cudaMalloc(&d_sink, sizeof(double)) != cudaSuccess) {
    cudaGetLastError();
    cudaFree(d_cyc);
    return VC_ERR_OOM;
  }
  cudaStream_t st = (cudaStream_t)stream;
  k_plcm_chain_latency<<<1, 32, 0, st>>>(x0, p, iters < 64 ? iters : 64, d_cyc, d_sink);  // warm-up
  k_plcm_chain_latency<<<1, 32, 0, st>>>(x0, p, iters, d_cyc, d_sink);
  long long cyc = 0;
  cudaError_t e = cudaMemcpyAsync(&cyc, d_cyc, sizeof(cyc), cudaMemcpyDeviceToHost, st);
  if (e == cudaSuccess) e = cudaStreamSynchronize(st);
  cudaFree(d_cyc);
  cudaFree(d_sink);
  if (e != cudaSuccess) return VC_ERR_CUDA;
  *cycles_per_step = (double)cyc / (double)((iters + 3) & ~3);
  return VC_OK;
}
