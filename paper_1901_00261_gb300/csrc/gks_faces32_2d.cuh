// gks_faces32_2d.cuh -- launch templates of the standalone 2D FP32-bulk sweeps, instantiated
// per reconstruction order in two translation units (gks_faces32.cu: 6th order,
// gks_faces32_o8.cu: 8th order) that compile in parallel.
#pragma once
#include <atomic>

#include "gks_sweep32.cuh"

namespace gks {

// Face rows per thread of the standalone 2D sweep tiles (TA32 x TB32 * FPT faces): linear
// Euler tiles SWEEP32_FPT; WENO-Z / viscous tiles SWEEP32_FPT_NX (x faces) and
// SWEEP32_FPT_NY (y faces).  The WENO-Z / viscous tiles run two blocks per SM, bound by
// registers, whatever their height, so their taller tiles cost no occupancy and an x-face
// tile reconstructs 1.25 slots per face instead of 1.5 (4096^2 shear layer, ms per step:
// 38.6 with 4 / 4 rows, 39.3 with 4 / 2, 40.0 with 2 / 2, 42.2 with 1 / 2).
#ifndef SWEEP32_FPT
#define SWEEP32_FPT 2
#endif
#ifndef SWEEP32_FPT_NX
#define SWEEP32_FPT_NX 4
#endif
#ifndef SWEEP32_FPT_NY
#define SWEEP32_FPT_NY 4
#endif

template <int ORDER, bool WENO, bool VISC, int DIR, bool WALLS, bool TANW>
inline cudaError_t launch_2d32_t(const FaceArgs32& a, cudaStream_t s) {
  constexpr int FPT = !(WENO || VISC) ? SWEEP32_FPT : (DIR == 0 ? SWEEP32_FPT_NX : SWEEP32_FPT_NY);
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
