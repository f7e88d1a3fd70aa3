// mgsa_fp64_probe: the FP64 fused multiply-add rate this GPU sustains, the
// denominator of the FP64 roofline fraction of the sweep kernels (declared in
// mgsa.h).  The paper has no counterpart: it is the measured ceiling the
// library's own kernels are compared against.
//
// Every thread runs kChains independent FMA chains, x <- x * a + b, so that
// the FP64 pipe, not the FMA latency, limits the rate.  With a = 1 - 2^-20 and
// b = 2^-20 every chain stays near 1 (no overflow, no denormals).  The chains'
// sum is stored so that the compiler keeps the work.
#include <cuda_runtime.h>

#include "mgsa.h"
#include "mgsa_internal.cuh"

namespace {

constexpr int kChains = 8;
constexpr int kProbeThreads = 256;
constexpr int kProbeCtasPerSm = 4;

__global__ void __launch_bounds__(kProbeThreads) dfma_probe_kernel(double* out, int iters, double a, double b) {
  double x[kChains];
#pragma unroll
  for (int c = 0; c < kChains; ++c) x[c] = 1.0 + 1e-3 * (double)(threadIdx.x + c);
  for (int it = 0; it < iters; ++it) {
#pragma unroll
    for (int c = 0; c < kChains; ++c) x[c] = fma(x[c], a, b);
  }
  double s = 0.0;
#pragma unroll
  for (int c = 0; c < kChains; ++c) s += x[c];
  out[blockIdx.x * (size_t)blockDim.x + threadIdx.x] = s;
}

}  // namespace

extern "C" mgsa_status mgsa_fp64_probe(int device, int iters, double* tflops, double* ms) {
  if (!tflops || !ms || iters < 1) {
    mgsa::set_last_error("mgsa_fp64_probe: NULL output or iters < 1");
    return MGSA_ERR_INVALID;
  }
  int prev = -1;
  if (cudaGetDevice(&prev) != cudaSuccess || cudaSetDevice(device) != cudaSuccess) {
    mgsa::set_last_error("mgsa_fp64_probe: bad device");
    return MGSA_ERR_INVALID;
  }
  int sms = 0;
  cudaError_t e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, device);
  const int grid = sms * kProbeCtasPerSm;
  double* out = nullptr;
  cudaEvent_t e0 = nullptr, e1 = nullptr;
  cudaStream_t s = nullptr;
  float t = 0.f;
  if (e == cudaSuccess) e = cudaMalloc(&out, sizeof(double) * (size_t)grid * kProbeThreads);
  if (e == cudaSuccess) e = cudaStreamCreateWithFlags(&s, cudaStreamNonBlocking);
  if (e == cudaSuccess) e = cudaEventCreate(&e0);
  if (e == cudaSuccess) e = cudaEventCreate(&e1);
  const double a = 1.0 - 1.0 / 1048576.0, b = 1.0 / 1048576.0;
  if (e == cudaSuccess) {  // one warm-up launch, then the timed one
    dfma_probe_kernel<<<grid, kProbeThreads, 0, s>>>(out, iters, a, b);
    e = cudaGetLastError();
  }
  if (e == cudaSuccess) e = cudaEventRecord(e0, s);
  if (e == cudaSuccess) {
    dfma_probe_kernel<<<grid, kProbeThreads, 0, s>>>(out, iters, a, b);
    e = cudaGetLastError();
  }
  if (e == cudaSuccess) e = cudaEventRecord(e1, s);
  if (e == cudaSuccess) e = cudaEventSynchronize(e1);
  if (e == cudaSuccess) e = cudaEventElapsedTime(&t, e0, e1);
  if (e0) cudaEventDestroy(e0);
  if (e1) cudaEventDestroy(e1);
  if (s) cudaStreamDestroy(s);
  if (out) cudaFree(out);
  if (prev >= 0) cudaSetDevice(prev);
  if (e != cudaSuccess) {
    mgsa::set_last_error(cudaGetErrorString(e));
    return MGSA_ERR_CUDA;
  }
  const double flops = 2.0 * kChains * (double)iters * (double)grid * kProbeThreads;
  *ms = (double)t;
  *tflops = flops / ((double)t * 1e-3) / 1e12;
  return MGSA_OK;
}
