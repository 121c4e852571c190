// Arithmetic-pipe throughput probe (no counterpart in the paper): the rates of
// the instructions the step's kernels are bound by, measured on the device in
// use -- FP64 FMA, FP32 FMA, FP64 -> FP32 conversion and FP64 comparison.
// Each kernel runs four independent dependency chains per thread over a grid
// of 8 blocks of 256 threads per multiprocessor; the conversion and
// comparison chains carry their dependency through integer operations, so the
// only FP64-pipe instruction of their loop is the one measured.
#include <cuda_runtime.h>

#include "../../include/adg.h"
#include "adg_internal.h"

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

// FP64 reciprocal by division (1.0 / x), four chains per thread; the next
// operand keeps the value near 1 with an integer change of its low word.
__global__ void probe_ddiv(double* out) {
  double x[4];
#pragma unroll
  for (int j = 0; j < 4; ++j) x[j] = threadIdx.x * 1e-3 + 1.0 + j;
  for (int i = 0; i < kIters; ++i)
#pragma unroll
    for (int j = 0; j < 4; ++j) {
      const double r = 1.0 / x[j];
      x[j] = __hiloint2double(__double2hiint(x[j]), __double2loint(x[j]) ^ (__double2loint(r) & 0xff));
    }
  out[blockIdx.x * blockDim.x + threadIdx.x] = x[0] + x[1] + x[2] + x[3];
}

// The same chains with rcp_newton.
__global__ void probe_rcpn(double* out) {
  double x[4];
#pragma unroll
  for (int j = 0; j < 4; ++j) x[j] = threadIdx.x * 1e-3 + 1.0 + j;
  for (int i = 0; i < kIters; ++i)
#pragma unroll
    for (int j = 0; j < 4; ++j) {
      const double r = adg::rcp_newton(x[j]);
      x[j] = __hiloint2double(__double2hiint(x[j]), __double2loint(x[j]) ^ (__double2loint(r) & 0xff));
    }
  out[blockIdx.x * blockDim.x + threadIdx.x] = x[0] + x[1] + x[2] + x[3];
}

// rcp_newton against 1.0 / x on 2^22 values: mantissas from a counter-based
// hash, exponents spanning 2^-60 .. 2^60 (inside the FP32 normal range), both
// signs.  acc[0]: largest difference in ulps of 1.0 / x; acc[1]: how many
// differ.
__global__ void check_rcpn(unsigned long long* acc) {
  const unsigned long long i = blockIdx.x * (unsigned long long)blockDim.x + threadIdx.x;
  unsigned long long h = i * 0x9E3779B97F4A7C15ull;
  h ^= h >> 31;
  h *= 0xBF58476D1CE4E5B9ull;
  h ^= h >> 29;
  const long long e = (long long)(i % 121) - 60 + 1023;
  const unsigned long long bits = ((i & 1ull) << 63) | ((unsigned long long)e << 52) | (h >> 12);
  const double x = __longlong_as_double((long long)bits);
  const double a = 1.0 / x, b = adg::rcp_newton(x);
  const long long d = __double_as_longlong(a) - __double_as_longlong(b);
  const unsigned long long ad = (unsigned long long)(d < 0 ? -d : d);
  if (ad) {
    atomicMax(&acc[0], ad);
    atomicAdd(&acc[1], 1ull);
  }
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
  void (*kernels[6])(double*) = {probe_dfma, probe_ffma, probe_d2f, probe_dsetp, probe_ddiv, probe_rcpn};
  const double per_thread[6] = {4.0 * kIters, 16.0 * kIters, 4.0 * kIters, 4.0 * kIters,
                                4.0 * kIters, 4.0 * kIters};
  const int nk = cap >= 6 ? 6 : 4;
  for (int k = 0; k < nk && rc == ADG_OK; ++k) {
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
  if (rc == ADG_OK && cap >= 8) {
    // the Newton reciprocal against the division
    unsigned long long* acc = nullptr;
    if (cudaMalloc(&acc, 2 * sizeof(unsigned long long)) != cudaSuccess) {
      rc = ADG_ERR_OOM;
    } else {
      unsigned long long h[2] = {0ull, 0ull};
      if (cudaMemset(acc, 0, sizeof(h)) != cudaSuccess) rc = ADG_ERR_CUDA;
      if (rc == ADG_OK) {
        check_rcpn<<<(1 << 22) / 256, 256>>>(acc);
        if (cudaGetLastError() != cudaSuccess ||
            cudaMemcpy(h, acc, sizeof(h), cudaMemcpyDeviceToHost) != cudaSuccess)
          rc = ADG_ERR_CUDA;
      }
      out[6] = (double)h[0];
      out[7] = (double)h[1] / (double)(1 << 22);
      cudaFree(acc);
    }
  }
  if (e0) cudaEventDestroy(e0);
  if (e1) cudaEventDestroy(e1);
  cudaFree(buf);
  return rc;
}
