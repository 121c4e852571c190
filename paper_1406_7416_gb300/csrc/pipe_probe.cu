// Arithmetic-pipe throughput probe (no counterpart in the paper): the rates of
// the instructions the step's kernels are bound by, measured on the device in
// use -- FP64 FMA, FP32 FMA, FP64 -> FP32 conversion and FP64 comparison.
// Each kernel runs four independent dependency chains per thread over a grid
// of 8 blocks of 256 threads per multiprocessor; the conversion and
// comparison chains carry their dependency through integer operations, so the
// only FP64-pipe instruction of their loop is the one measured.
#include <cuda_runtime.h>

#include "../../include/adg.h"

namespace {

constexpr int kIters = 4096;

__global__ void probe_dfma(double* out) {
  const double b = 1.0000001, c = 1e-7;
  double x0 = threadIdx.x * 1e-3 + 1.0, x1 = x0 + 1.0, x2 = x0 + 2.0, x3 = x0 + 3.0;
  for (int i = 0; i < kIters; ++i) {
    x0 = fma(x0, b, c);
    x1 = fma(x1, b, c);
    x2 = fma(x2, b, c);
    x3 = fma(x3, b, c);
  }
  out[blockIdx.x * blockDim.x + threadIdx.x] = x0 + x1 + x2 + x3;
}

__global__ void probe_ffma(double* out) {
  const float b = 1.0000001f, c = 1e-7f;
  float x[16];
#pragma unroll
  for (int j = 0; j < 16; ++j) x[j] = threadIdx.x * 1e-3f + j;
  for (int i = 0; i < kIters; ++i)
#pragma unroll
    for (int j = 0; j < 16; ++j) x[j] = fmaf(x[j], b, c);
  float s = 0.0f;
#pragma unroll
  for (int j = 0; j < 16; ++j) s += x[j];
  out[blockIdx.x * blockDim.x + threadIdx.x] = s;
}

__global__ void probe_d2f(double* out) {
  double x[4];
#pragma unroll
  for (int j = 0; j < 4; ++j) x[j] = threadIdx.x * 1e-3 + 1.0 + j;
  for (int i = 0; i < kIters; ++i)
#pragma unroll
    for (int j = 0; j < 4; ++j)
      x[j] = __hiloint2double(__double2hiint(x[j]), __double2loint(x[j]) ^ __float_as_int((float)x[j]));
  out[blockIdx.x * blockDim.x + threadIdx.x] = x[0] + x[1] + x[2] + x[3];
}

__global__ void probe_dsetp(double* out) {
  double x[4];
#pragma unroll
  for (int j = 0; j < 4; ++j) x[j] = threadIdx.x * 1e-3 + 1.0 + j;
  int c = 0;
  for (int i = 0; i < kIters; ++i) {
#pragma unroll
    for (int j = 0; j < 4; ++j) c += x[j] > 1.5 + j;
#pragma unroll
    for (int j = 0; j < 4; ++j) x[j] = __hiloint2double(__double2hiint(x[j]), __double2loint(x[j]) ^ (c & 7));
  }
  out[blockIdx.x * blockDim.x + threadIdx.x] = x[0] + x[1] + x[2] + x[3] + c;
}

}  // namespace

extern "C" int adg_pipe_rates(double* out, int cap) {
  if (!out || cap < 4) return ADG_ERR_ARG;
  int dev = 0, sms = 0;
  if (cudaGetDevice(&dev) != cudaSuccess ||
      cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess)
    return ADG_ERR_CUDA;
  const int blocks = sms * 8, threads = 256;
  double* buf = nullptr;
  if (cudaMalloc(&buf, sizeof(double) * blocks * threads) != cudaSuccess) return ADG_ERR_OOM;
  cudaEvent_t e0 = nullptr, e1 = nullptr;
  int rc = ADG_OK;
  if (cudaEventCreate(&e0) != cudaSuccess || cudaEventCreate(&e1) != cudaSuccess) rc = ADG_ERR_CUDA;
  void (*kernels[4])(double*) = {probe_dfma, probe_ffma, probe_d2f, probe_dsetp};
  const double per_thread[4] = {4.0 * kIters, 16.0 * kIters, 4.0 * kIters, 4.0 * kIters};
  for (int k = 0; k < 4 && rc == ADG_OK; ++k) {
    float best = 0.0f;
    for (int rep = 0; rep < 3 && rc == ADG_OK; ++rep) {
      float ms = 0.0f;
      if (cudaEventRecord(e0) != cudaSuccess) rc = ADG_ERR_CUDA;
      kernels[k]<<<blocks, threads>>>(buf);
      if (rc == ADG_OK && (cudaGetLastError() != cudaSuccess || cudaEventRecord(e1) != cudaSuccess ||
                           cudaEventSynchronize(e1) != cudaSuccess ||
                           cudaEventElapsedTime(&ms, e0, e1) != cudaSuccess))
        rc = ADG_ERR_CUDA;
      if (rep > 0 && (best == 0.0f || ms < best)) best = ms;   // the first run warms up
    }
    // thread operations per second (FMA: two flop each)
    if (rc == ADG_OK) out[k] = per_thread[k] * blocks * threads / (best * 1e-3);
  }
  if (e0) cudaEventDestroy(e0);
  if (e1) cudaEventDestroy(e1);
  cudaFree(buf);
  return rc;
}
