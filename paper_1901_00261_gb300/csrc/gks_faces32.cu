// gks_faces32.cu -- standalone launches of the FP32-bulk sweeps and updates (gks_sweep32.cuh).
#include "gks_faces32_2d.cuh"

namespace gks {

cudaError_t launch_mirror(const double* S, float* M, int nx, int ny, int dim, cudaStream_t s) {
  return launch_mirror_rows(S, M, nx, ny, dim, 0, ny, s);
}

cudaError_t launch_mirror_rows(const double* S, float* M, int nx, int ny, int dim, int j0, int nrows,
                               cudaStream_t s) {
  const long ncell = (long)nx * ny, c0 = (long)j0 * nx, n = (long)nrows * nx;
  if (n <= 0) return cudaSuccess;
  unsigned blocks = (unsigned)((n + 255) / 256);
  if (dim == 1) mirror_kernel<1><<<blocks, 256, 0, s>>>(S, M, ncell, c0, n);
  else mirror_kernel<2><<<blocks, 256, 0, s>>>(S, M, ncell, c0, n);
  return cudaGetLastError();
}

// ---------------------------------------------------------------------------
// Launchers
// ---------------------------------------------------------------------------
// Grids with a reflecting wall run the instantiations compiled with the wall signs.
template <int ORDER, bool WENO, bool VISC>
static cudaError_t launch_1d32_t(const FaceArgs32& a, cudaStream_t s) {
  int threads = 128;
  int blocks = (a.nx + 1 + threads - 1) / threads;
  const bool walls = a.bcx == 2;
  if (a.stage == 1) {
    if (walls) faces_1d_f32_kernel<ORDER, WENO, VISC, 1, true><<<blocks, threads, 0, s>>>(a);
    else faces_1d_f32_kernel<ORDER, WENO, VISC, 1, false><<<blocks, threads, 0, s>>>(a);
  } else {
    if (walls) faces_1d_f32_kernel<ORDER, WENO, VISC, 2, true><<<blocks, threads, 0, s>>>(a);
    else faces_1d_f32_kernel<ORDER, WENO, VISC, 2, false><<<blocks, threads, 0, s>>>(a);
  }
  return cudaGetLastError();
}

cudaError_t launch_faces32_1d(const FaceArgs32& a, int order, int recon, bool visc, cudaStream_t s) {
  if (order == 6) {
    if (recon == 0) return visc ? launch_1d32_t<6, false, true>(a, s) : launch_1d32_t<6, false, false>(a, s);
    return visc ? launch_1d32_t<6, true, true>(a, s) : launch_1d32_t<6, true, false>(a, s);
  }
  if (recon == 0) return visc ? launch_1d32_t<8, false, true>(a, s) : launch_1d32_t<8, false, false>(a, s);
  return visc ? launch_1d32_t<8, true, true>(a, s) : launch_1d32_t<8, true, false>(a, s);
}

cudaError_t launch_faces32_2d(const FaceArgs32& a, int dir, int order, int recon, bool visc, cudaStream_t s) {
  if (order == 6) return launch_faces32_2d_order<6>(a, dir, recon, visc, s);
  return launch_faces32_2d_o8(a, dir, recon, visc, s);
}

__global__ void rcp64_probe_kernel(const double* x, int n, double* out) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n) out[i] = rcp64(x[i]);
}

__global__ void d2f_probe_kernel(const double* x, int n, float* out) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n) out[i] = d2f_int(x[i]);
}

// d2f_int of host x[0..n) into host out[0..n); synchronous (test probe).
cudaError_t probe_d2f(const double* x, int n, float* out) {
  double* d = nullptr;
  float* o = nullptr;
  cudaError_t e = cudaMalloc(&d, (size_t)n * sizeof(double));
  if (e == cudaSuccess) e = cudaMalloc(&o, (size_t)n * sizeof(float));
  if (e == cudaSuccess) e = cudaMemcpy(d, x, (size_t)n * sizeof(double), cudaMemcpyHostToDevice);
  if (e == cudaSuccess) {
    d2f_probe_kernel<<<(n + 127) / 128, 128>>>(d, n, o);
    e = cudaGetLastError();
  }
  if (e == cudaSuccess) e = cudaMemcpy(out, o, (size_t)n * sizeof(float), cudaMemcpyDeviceToHost);
  if (d) cudaFree(d);
  if (o) cudaFree(o);
  return e;
}

// rcp64 of host x[0..n) into host out[0..n); synchronous (test probe).
cudaError_t probe_rcp64(const double* x, int n, double* out) {
  double* d = nullptr;
  cudaError_t e = cudaMalloc(&d, 2 * (size_t)n * sizeof(double));
  if (e != cudaSuccess) return e;
  e = cudaMemcpy(d, x, (size_t)n * sizeof(double), cudaMemcpyHostToDevice);
  if (e == cudaSuccess) {
    rcp64_probe_kernel<<<(n + 127) / 128, 128>>>(d, n, d + n);
    e = cudaGetLastError();
  }
  if (e == cudaSuccess) e = cudaMemcpy(out, d + n, (size_t)n * sizeof(double), cudaMemcpyDeviceToHost);
  cudaFree(d);
  return e;
}

cudaError_t launch_update32(const UpdateArgs32& a, int dim, int stage, cudaStream_t s) {
  long ncell = (long)a.nx * a.ny;
  unsigned blocks = (unsigned)((ncell + 255) / 256);
  if (dim == 1) {
    if (stage == 1) update_f32_kernel<1, 1><<<blocks, 256, 0, s>>>(a);
    else update_f32_kernel<1, 2><<<blocks, 256, 0, s>>>(a);
  } else {
    if (stage == 1) update_f32_kernel<2, 1><<<blocks, 256, 0, s>>>(a);
    else update_f32_kernel<2, 2><<<blocks, 256, 0, s>>>(a);
  }
  return cudaGetLastError();
}

}  // namespace gks
