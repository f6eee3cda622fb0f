// FP64 FMA throughput of the current GPU: the denominator of the FP64 step's
// roofline.  With FP64 storage the step is bound by the FP64 arithmetic pipe,
// not by HBM (GB300 keeps only a narrow FP64 pipe per SM), so its rate is
// reported against this measured peak.
//
// Every thread runs CHAINS independent FMA chains (enough to hide the pipe's
// latency with a few warps per scheduler) for a fixed number of iterations;
// the grid is BLOCKS_PER_SM blocks of 256 threads per SM.  The launch is timed
// with CUDA events on the caller's stream; the best of a few launches is kept.
#include <cuda_runtime.h>

#include <string>

#include "olb.h"
#include "olb_internal.h"

namespace {

constexpr int PK_NT = 256;
constexpr int CHAINS = 8;
constexpr int BLOCKS_PER_SM = 4;

__global__ void __launch_bounds__(PK_NT) fp64_fma_kernel(double* sink, int iters, double a, double b) {
  double x[CHAINS];
#pragma unroll
  for (int k = 0; k < CHAINS; ++k) x[k] = 1e-3 * threadIdx.x + k;
  for (int it = 0; it < iters; ++it) {
#pragma unroll
    for (int k = 0; k < CHAINS; ++k) x[k] = fma(x[k], a, b);
  }
  double s = 0.0;
#pragma unroll
  for (int k = 0; k < CHAINS; ++k) s += x[k];
  // never true for the arguments used; keeps every chain live
  if (s == -1.0) sink[blockIdx.x] = s;
}

int fail(int code, const std::string& m) {
  olb::set_last_error(m);
  return code;
}

}  // namespace

extern "C" int olb_fp64_fma_peak(void* stream, double* flops_per_s) {
  if (!flops_per_s) return fail(OLB_EINVAL, "null output");
  int dev = 0, sms = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e == cudaSuccess) e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  if (e != cudaSuccess) return fail(OLB_ECUDA, std::string("device query: ") + cudaGetErrorString(e));
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  const int blocks = sms * BLOCKS_PER_SM;
  const int iters = 20000;  // about 30 ms at 1.25 TFLOP/s on 152 SMs
  double* sink = nullptr;
  cudaEvent_t t0 = nullptr, t1 = nullptr;
  e = cudaMallocAsync(&sink, sizeof(double) * blocks, s);
  if (e == cudaSuccess) e = cudaEventCreate(&t0);
  if (e == cudaSuccess) e = cudaEventCreate(&t1);
  float best_ms = 0.f;
  for (int rep = 0; rep < 4 && e == cudaSuccess; ++rep) {  // the first launch is a warm-up
    cudaEventRecord(t0, s);
    fp64_fma_kernel<<<blocks, PK_NT, 0, s>>>(sink, iters, 0.999999, 1e-6);
    e = cudaGetLastError();
    cudaEventRecord(t1, s);
    if (e == cudaSuccess) e = cudaEventSynchronize(t1);
    float ms = 0.f;
    if (e == cudaSuccess) e = cudaEventElapsedTime(&ms, t0, t1);
    if (e == cudaSuccess && rep > 0 && (best_ms == 0.f || ms < best_ms)) best_ms = ms;
  }
  if (sink) cudaFreeAsync(sink, s);
  if (t0) cudaEventDestroy(t0);
  if (t1) cudaEventDestroy(t1);
  if (e != cudaSuccess) return fail(OLB_ECUDA, std::string("FP64 peak kernel: ") + cudaGetErrorString(e));
  if (!(best_ms > 0.f)) return fail(OLB_ECUDA, "FP64 peak kernel: no timing");
  const double fmas = (double)blocks * PK_NT * iters * CHAINS;
  *flops_per_s = 2.0 * fmas / (best_ms * 1e-3);
  return OLB_OK;
}
