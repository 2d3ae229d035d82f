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

template <int ORDER, bool WENO, bool VISC, int DIR, bool WALLS>
static cudaError_t launch_2d32_t(const FaceArgs32& a, cudaStream_t s) {
  const int FPT = SWEEP32_FPT;
  typedef Tile32<DIR, FPT> T;
  const size_t shmem = T::smem_bytes(WENO);
  static bool attr_set = false;
  if (!attr_set) {
    cudaError_t e = cudaFuncSetAttribute(faces_2d_f32_kernel<ORDER, WENO, VISC, DIR, FPT, 1, WALLS>,
                                         cudaFuncAttributeMaxDynamicSharedMemorySize, (int)shmem);
    if (e == cudaSuccess)
      e = cudaFuncSetAttribute(faces_2d_f32_kernel<ORDER, WENO, VISC, DIR, FPT, 2, WALLS>,
                               cudaFuncAttributeMaxDynamicSharedMemorySize, (int)shmem);
    if (e != cudaSuccess) return e;
    attr_set = true;
  }
  dim3 block(TA32, TB32);
  dim3 grid;
  if (DIR == 0) grid = dim3((a.nx + 1 + TA32 - 1) / TA32, (a.ny + T::TB - 1) / T::TB);
  else grid = dim3((a.nx + TA32 - 1) / TA32, (a.ny + 1 + T::TB - 1) / T::TB);
  if (a.stage == 1) faces_2d_f32_kernel<ORDER, WENO, VISC, DIR, FPT, 1, WALLS><<<grid, block, shmem, s>>>(a);
  else faces_2d_f32_kernel<ORDER, WENO, VISC, DIR, FPT, 2, WALLS><<<grid, block, shmem, s>>>(a);
  return cudaGetLastError();
}

template <int ORDER, bool WENO, bool VISC>
static cudaError_t launch_2d32_dir(const FaceArgs32& a, int dir, cudaStream_t s) {
  const bool walls = a.bcx == 2 || a.bcy == 2;
  if (walls)
    return dir == 0 ? launch_2d32_t<ORDER, WENO, VISC, 0, true>(a, s) : launch_2d32_t<ORDER, WENO, VISC, 1, true>(a, s);
  return dir == 0 ? launch_2d32_t<ORDER, WENO, VISC, 0, false>(a, s) : launch_2d32_t<ORDER, WENO, VISC, 1, false>(a, s);
}

cudaError_t launch_faces32_2d(const FaceArgs32& a, int dir, int order, int recon, bool visc, cudaStream_t s) {
  if (order == 6) {
    if (recon == 0) return visc ? launch_2d32_dir<6, false, true>(a, dir, s) : launch_2d32_dir<6, false, false>(a, dir, s);
    return visc ? launch_2d32_dir<6, true, true>(a, dir, s) : launch_2d32_dir<6, true, false>(a, dir, s);
  }
  if (recon == 0) return visc ? launch_2d32_dir<8, false, true>(a, dir, s) : launch_2d32_dir<8, false, false>(a, dir, s);
  return visc ? launch_2d32_dir<8, true, true>(a, dir, s) : launch_2d32_dir<8, true, false>(a, dir, s);
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
