// gks_probe.cu -- arithmetic-throughput probe used as the roofline denominator of the
// ALU-bound face sweeps (independent FMA chains in every thread of a full grid), and a probe
// that evaluates the face kernels' FP64 time-integration coefficients for tests.
#include <cuda_runtime.h>

#include "gks_device.cuh"

namespace gks {

// time_coefs(theta, 1/(2 theta), dt) for theta[i], as the non-equilibrium branch of the face
// kernels forms it (SINGLE: the single-precision form's truncation); out[4 i ..] = a0, a1, b0,
// b1.
template <bool SINGLE>
__global__ void time_coefs_probe_kernel(const double* theta, int n, double dt, double* out) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  const double th = theta[i];
  const TimeCoef T = time_coefs<SINGLE>(th, 0.5 / th, dt);
  out[4 * i + 0] = T.a0;
  out[4 * i + 1] = T.a1;
  out[4 * i + 2] = T.b0;
  out[4 * i + 3] = T.b1;
}

// Host arrays theta[n] and out[4 n]; synchronous.
cudaError_t probe_time_coefs(const double* theta, int n, double dt, double* out, bool single) {
  double* d_theta = nullptr;
  double* d_out = nullptr;
  cudaError_t e = cudaMalloc(&d_theta, (size_t)n * sizeof(double));
  if (e == cudaSuccess) e = cudaMalloc(&d_out, (size_t)n * 4 * sizeof(double));
  if (e == cudaSuccess) e = cudaMemcpy(d_theta, theta, (size_t)n * sizeof(double), cudaMemcpyHostToDevice);
  if (e == cudaSuccess) {
    if (single) time_coefs_probe_kernel<true><<<(n + 127) / 128, 128>>>(d_theta, n, dt, d_out);
    else time_coefs_probe_kernel<false><<<(n + 127) / 128, 128>>>(d_theta, n, dt, d_out);
    e = cudaGetLastError();
  }
  if (e == cudaSuccess) e = cudaMemcpy(out, d_out, (size_t)n * 4 * sizeof(double), cudaMemcpyDeviceToHost);
  if (d_theta) cudaFree(d_theta);
  if (d_out) cudaFree(d_out);
  return e;
}

template <typename T>
__global__ void __launch_bounds__(256) fma_probe_kernel(T* out, int iters, T a, T b) {
  T x0 = T(threadIdx.x) * T(1e-3), x1 = x0 + T(1), x2 = x0 + T(2), x3 = x0 + T(3);
  T x4 = x0 + T(4), x5 = x0 + T(5), x6 = x0 + T(6), x7 = x0 + T(7);
  for (int i = 0; i < iters; ++i) {
    x0 = fma(x0, a, b); x1 = fma(x1, a, b); x2 = fma(x2, a, b); x3 = fma(x3, a, b);
    x4 = fma(x4, a, b); x5 = fma(x5, a, b); x6 = fma(x6, a, b); x7 = fma(x7, a, b);
  }
  T s = x0 + x1 + x2 + x3 + x4 + x5 + x6 + x7;
  if (s == T(-12345)) out[blockIdx.x] = s;   // keeps the chains alive
}

// FLOP/s (2 per FMA) of the probe; fp64 != 0 selects double.
cudaError_t probe_fma(int fp64, int iters, double* flops, cudaStream_t s) {
  int dev = 0, sms = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e == cudaSuccess) e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  if (e != cudaSuccess) return e;
  const int blocks = sms * 8, threads = 256;
  void* out = nullptr;
  e = cudaMalloc(&out, blocks * sizeof(double));
  if (e != cudaSuccess) return e;
  cudaEvent_t t0, t1;
  cudaEventCreate(&t0); cudaEventCreate(&t1);
  float best = 1e30f;
  for (int rep = 0; rep < 4; ++rep) {
    cudaEventRecord(t0, s);
    if (fp64) fma_probe_kernel<double><<<blocks, threads, 0, s>>>((double*)out, iters, 0.999999, 1e-7);
    else fma_probe_kernel<float><<<blocks, threads, 0, s>>>((float*)out, iters, 0.999999f, 1e-7f);
    cudaEventRecord(t1, s);
    e = cudaEventSynchronize(t1);
    if (e != cudaSuccess) break;
    float ms = 0;
    cudaEventElapsedTime(&ms, t0, t1);
    if (rep > 0 && ms < best) best = ms;   // first launch is a warm-up
  }
  if (e == cudaSuccess) e = cudaGetLastError();
  cudaEventDestroy(t0); cudaEventDestroy(t1);
  cudaFree(out);
  if (e != cudaSuccess) return e;
  *flops = 2.0 * 8.0 * (double)iters * blocks * threads / (best * 1e-3);
  return cudaSuccess;
}

}  // namespace gks
