// gks_kernels.cuh -- kernel declarations shared by the launch units and the C-ABI.
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>

#include "gks_device.cuh"

namespace gks {

// Status bits written by kernels (read back by the host at synchronising calls).
enum : unsigned int { ST_NONPHYSICAL = 1u, ST_NONFINITE = 2u };

// One face sweep (one direction, one stage).
struct FaceArgs {
  const double* W;     // [nv][ny][nx] conservative cell averages
  const double* Wn;    // [nv][ny][nx] cell-averaged gradient along the face normal
  double* out;         // [ncomp][nv][nfaces] face results (layout per direction below)
  const double* dtp;   // device scalar dt
  unsigned int* status;
  int nx, ny;          // cells
  int bcx, bcy;        // 0 periodic, 1 transmissive
  double dn, dtan;     // cell size along the normal / tangential direction
  int stage;           // 1 or 2
  PhysParams P;
};

// Cell update after the face sweeps of a stage.
struct UpdateArgs {
  const double* W;      // state of the stage's data (Wn for stage 1)
  const double* fx;     // x-face buffer [ncomp][nv][ny][nx+1]
  const double* fy;     // y-face buffer [ncomp][nv][ny+1][nx] (2D)
  double* Ws;           // stage 1: W*, Wx*, Wy* (3 planes-sets); stage 2: Wn+1 output
  double* acc;          // accumulators (W, Wx, Wy)
  int nx, ny;
  double idx, idy;
};

// launchers (defined in the .cu units)
cudaError_t launch_faces_1d(const FaceArgs& a, int order, int recon, bool visc, cudaStream_t s);
cudaError_t launch_faces_2d(const FaceArgs& a, int dir, int order, int recon, bool visc, cudaStream_t s);
cudaError_t launch_update(const UpdateArgs& a, int dim, int stage, cudaStream_t s);
cudaError_t launch_wavespeed(const double* W, int nx, int ny, int dim, double gamma, double dx,
                             double dy, unsigned long long* out, cudaStream_t s);
cudaError_t launch_set_scalar(double* p, double v, cudaStream_t s);
cudaError_t probe_fma(int fp64, int iters, double* flops, cudaStream_t s);

}  // namespace gks
