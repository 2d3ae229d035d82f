// gks_faces32_2d.cuh -- launch templates of the standalone 2D FP32-bulk sweeps, instantiated
// per reconstruction order in two translation units (gks_faces32.cu: 6th order,
// gks_faces32_o8.cu: 8th order) that compile in parallel.
#pragma once
#include <atomic>

#include "gks_sweep32.cuh"

namespace gks {

// Face rows per thread of the standalone 2D sweep tiles (TA32 x TB32 * SWEEP32_FPT faces).
#ifndef SWEEP32_FPT
#define SWEEP32_FPT 2
#endif

template <int ORDER, bool WENO, bool VISC, int DIR, bool WALLS, bool TANW>
inline cudaError_t launch_2d32_t(const FaceArgs32& a, cudaStream_t s) {
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
inline cudaError_t launch_2d32_tw(const FaceArgs32& a, int dir, cudaStream_t s) {
  if (WENO && a.P.tan_mode == 1)
    return dir == 0 ? launch_2d32_t<ORDER, WENO, VISC, 0, WALLS, WENO>(a, s)
                    : launch_2d32_t<ORDER, WENO, VISC, 1, WALLS, WENO>(a, s);
  return dir == 0 ? launch_2d32_t<ORDER, WENO, VISC, 0, WALLS, false>(a, s)
                  : launch_2d32_t<ORDER, WENO, VISC, 1, WALLS, false>(a, s);
}

template <int ORDER, bool WENO, bool VISC>
inline cudaError_t launch_2d32_dir(const FaceArgs32& a, int dir, cudaStream_t s) {
  const bool walls = a.bcx == 2 || a.bcy == 2;
  if (walls) return launch_2d32_tw<ORDER, WENO, VISC, true>(a, dir, s);
  return launch_2d32_tw<ORDER, WENO, VISC, false>(a, dir, s);
}

// All 2D sweeps of reconstruction order ORDER.
template <int ORDER>
cudaError_t launch_faces32_2d_order(const FaceArgs32& a, int dir, int recon, bool visc, cudaStream_t s) {
  if (recon == 0) return visc ? launch_2d32_dir<ORDER, false, true>(a, dir, s) : launch_2d32_dir<ORDER, false, false>(a, dir, s);
  return visc ? launch_2d32_dir<ORDER, true, true>(a, dir, s) : launch_2d32_dir<ORDER, true, false>(a, dir, s);
}

// defined in gks_faces32_o8.cu
cudaError_t launch_faces32_2d_o8(const FaceArgs32& a, int dir, int recon, bool visc, cudaStream_t s);

}  // namespace gks
