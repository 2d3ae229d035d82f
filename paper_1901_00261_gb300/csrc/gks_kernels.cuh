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

// FP32-bulk face sweep: reads the FP32 mirror of the state, writes FP32 deltas.
struct FaceArgs32 {
  const float* M;      // mirror [hi (nv planes) | lo (nv planes) | ...]
  const float* Mn;     // mirrored gradient along the face normal [nv][ny][nx]
  const double* fref;  // per-cell FP64 Euler fluxes [F | G][nv][ncell]
  void* out;           // face buffer (FP64 planes, then FP32 planes)
  const double* dtp;
  unsigned int* status;
  int nx, ny, bcx, bcy;
  double dn, dtan;
  float dnf, itanf, gammaf, epsf;   // single-precision copies (dn, 1/dtan, gamma, WENO eps)
  int stage;
  PhysParams P;
};

// FP32-bulk cell update: FP64 accumulation; writes the next mirror.
struct UpdateArgs32 {
  const double* W;     // FP64 state W^n (stage 1)
  const float* fx;
  const float* fy;
  double* Ws;
  double* acc;
  float* M;            // mirror written for the next sweep
  double* fref;        // per-cell FP64 Euler fluxes [F | G][nv][ncell] of the step's state
  const double* dtp;
  int nx, ny, bcx, bcy;
  double idx, idy, gamma;
};

// launchers (defined in the .cu units)
cudaError_t launch_mirror_ref(const double* S, float* M, double* fref, int nx, int ny, int dim,
                              double gamma, cudaStream_t s);
cudaError_t launch_faces32_1d(const FaceArgs32& a, int order, int recon, bool visc, cudaStream_t s);
cudaError_t launch_faces32_2d(const FaceArgs32& a, int dir, int order, int recon, bool visc, cudaStream_t s);
cudaError_t launch_update32(const UpdateArgs32& a, int dim, int stage, cudaStream_t s);
cudaError_t launch_faces_1d(const FaceArgs& a, int order, int recon, bool visc, cudaStream_t s);
cudaError_t launch_faces_2d(const FaceArgs& a, int dir, int order, int recon, bool visc, cudaStream_t s);
cudaError_t launch_update(const UpdateArgs& a, int dim, int stage, cudaStream_t s);
cudaError_t launch_wavespeed(const double* W, int nx, int ny, int dim, double gamma, double dx,
                             double dy, unsigned long long* out, cudaStream_t s);
cudaError_t launch_set_scalar(double* p, double v, cudaStream_t s);
cudaError_t probe_fma(int fp64, int iters, double* flops, cudaStream_t s);

}  // namespace gks
