// gks_faces32.cu -- standalone launches of the FP32-bulk sweeps and updates (gks_sweep32.cuh).
#include "gks_sweep32.cuh"

namespace gks {

cudaError_t launch_mirror(const double* S, float* M, int nx, int ny, int dim, cudaStream_t s) {
  long ncell = (long)nx * ny;
  unsigned blocks = (unsigned)((ncell + 255) / 256);
  if (dim == 1) mirror_kernel<1><<<blocks, 256, 0, s>>>(S, M, ncell);
  else mirror_kernel<2><<<blocks, 256, 0, s>>>(S, M, ncell);
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

// Face rows per thread of the standalone 2D sweep tiles (TA32 x TB32 * SWEEP32_FPT faces).
#ifndef SWEEP32_FPT
#define SWEEP32_FPT 2
#endif

template <int ORDER, bool WENO, bool VISC, int DIR, bool WALLS, bool TANW>
static cudaError_t launch_2d32_t(const FaceArgs32& a, cudaStream_t s) {
  const int FPT = SWEEP32_FPT;
  typedef Tile32<DIR, FPT> T;
  const size_t shmem = T::smem_bytes(WENO);
  static std::atomic<unsigned long long> smem_set{0};
  const void* fns[2] = {(const void*)faces_2d_f32_kernel<ORDER, WENO, VISC, DIR, FPT, 1, WALLS, TANW>,
                        (const void*)faces_2d_f32_kernel<ORDER, WENO, VISC, DIR, FPT, 2, WALLS, TANW>};
  cudaError_t e = smem_limit_per_device(smem_set, fns, 2, (int)shmem);
  if (e != cudaSuccess) return e;
  dim3 block(TA32, TB32);
  dim3 grid;
  if (DIR == 0) grid = dim3((a.nx + 1 + TA32 - 1) / TA32, (a.ny + T::TB - 1) / T::TB);
  else grid = dim3((a.nx + TA32 - 1) / TA32, (a.ny + 1 + T::TB - 1) / T::TB);
  if (a.stage == 1) faces_2d_f32_kernel<ORDER, WENO, VISC, DIR, FPT, 1, WALLS, TANW><<<grid, block, shmem, s>>>(a);
  else faces_2d_f32_kernel<ORDER, WENO, VISC, DIR, FPT, 2, WALLS, TANW><<<grid, block, shmem, s>>>(a);
  return cudaGetLastError();
}

// tan_mode 1 (tangential WENO-Z) selects separate instantiations of the WENO-Z tiles, so that
// the default tiles carry none of its code or registers
template <int ORDER, bool WENO, bool VISC, bool WALLS>
static cudaError_t launch_2d32_tw(const FaceArgs32& a, int dir, cudaStream_t s) {
  if (WENO && a.P.tan_mode == 1)
    return dir == 0 ? launch_2d32_t<ORDER, WENO, VISC, 0, WALLS, WENO>(a, s)
                    : launch_2d32_t<ORDER, WENO, VISC, 1, WALLS, WENO>(a, s);
  return dir == 0 ? launch_2d32_t<ORDER, WENO, VISC, 0, WALLS, false>(a, s)
                  : launch_2d32_t<ORDER, WENO, VISC, 1, WALLS, false>(a, s);
}

template <int ORDER, bool WENO, bool VISC>
static cudaError_t launch_2d32_dir(const FaceArgs32& a, int dir, cudaStream_t s) {
  const bool walls = a.bcx == 2 || a.bcy == 2;
  if (walls) return launch_2d32_tw<ORDER, WENO, VISC, true>(a, dir, s);
  return launch_2d32_tw<ORDER, WENO, VISC, false>(a, dir, s);
}

cudaError_t launch_faces32_2d(const FaceArgs32& a, int dir, int order, int recon, bool visc, cudaStream_t s) {
  if (order == 6) {
    if (recon == 0) return visc ? launch_2d32_dir<6, false, true>(a, dir, s) : launch_2d32_dir<6, false, false>(a, dir, s);
    return visc ? launch_2d32_dir<6, true, true>(a, dir, s) : launch_2d32_dir<6, true, false>(a, dir, s);
  }
  if (recon == 0) return visc ? launch_2d32_dir<8, false, true>(a, dir, s) : launch_2d32_dir<8, false, false>(a, dir, s);
  return visc ? launch_2d32_dir<8, true, true>(a, dir, s) : launch_2d32_dir<8, true, false>(a, dir, s);
}

__global__ void rcp64_probe_kernel(const double* x, int n, double* out) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n) out[i] = rcp64(x[i]);
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
