// gks_kernels.cuh -- kernel declarations shared by the launch units and the C-ABI.
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>

#include <atomic>

#include "gks_device.cuh"

namespace gks {

// Raise the dynamic shared-memory limit of kernels fns[0..n) to `bytes` on the current
// device, once per device: function attributes belong to a device, so each device that
// launches the kernels needs its own setting.  `done` holds one bit per device (devices
// 64 and above set the attribute on every call).  Setting it twice is harmless, so two host
// threads that race on the first launch both set it.
inline cudaError_t smem_limit_per_device(std::atomic<unsigned long long>& done,
                                         const void* const* fns, int n, int bytes) {
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return e;
  const unsigned long long bit = dev < 64 ? (1ull << dev) : 0ull;
  if (bit && (done.load(std::memory_order_acquire) & bit)) return cudaSuccess;
  for (int i = 0; i < n; ++i) {
    e = cudaFuncSetAttribute(fns[i], cudaFuncAttributeMaxDynamicSharedMemorySize, bytes);
    if (e != cudaSuccess) return e;
  }
  if (bit) done.fetch_or(bit, std::memory_order_release);
  return cudaSuccess;
}

// Status bits written by kernels (read back by the host at synchronising calls).
enum : unsigned int { ST_NONPHYSICAL = 1u, ST_NONFINITE = 2u };

// Time constants of a step, derived from dt once per change of dt (dt first, so a kernel
// that needs only dt reads the first double).  The MSMD weights of Sec. 2.3: dt/2 and
// dt^2/8 (W*), dt and dt^2/6 (W^{n+1}, stage 1), dt^2/3 (stage 2).
struct StepTimes {
  double dt, h, h2, s6, s3;
  float dtf, hf, h2f, s6f, s3f, pad[3];
};
static_assert(sizeof(StepTimes) == 72, "StepTimes layout");
constexpr int STEP_TIMES_DOUBLES = 9;   // storage of one StepTimes in doubles

__host__ __device__ inline StepTimes step_times(double dt) {
  StepTimes T;
  const double dt2 = dt * dt;
  T.dt = dt; T.h = 0.5 * dt; T.h2 = 0.125 * dt2; T.s6 = dt2 * (1.0 / 6.0); T.s3 = dt2 * (1.0 / 3.0);
  T.dtf = (float)T.dt; T.hf = (float)T.h; T.h2f = (float)T.h2; T.s6f = (float)T.s6; T.s3f = (float)T.s3;
  T.pad[0] = T.pad[1] = T.pad[2] = 0.f;
  return T;
}

// One face sweep (one direction, one stage).
struct FaceArgs {
  const double* W;     // [nv][ny][nx] conservative cell averages
  const double* Wn;    // [nv][ny][nx] cell-averaged gradient along the face normal
  double* out;         // [ncomp][nv][nfaces] face results (layout per direction below)
  const double* dtp;   // device scalar dt
  unsigned int* status;
  int nx, ny;          // cells
  int bcx, bcy;        // 0 periodic, 1 transmissive, 2 reflecting wall, 3 isothermal wall
  double dn, dtan;     // cell size along the normal / tangential direction
  int stage;           // 1 or 2
  PhysParams P;
  double wallT[4], wallU[4];   // isothermal walls at x0, x1, y0, y1: p/rho, tangential velocity
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
  const double* W;     // FP64 state [nv][ny][nx] (stage 1: reference fluxes and cell differences)
  void* out;           // face buffer (one FP64 block, then five FP32 blocks; see ld_face64)
  const double* dtp;
  unsigned int* status;
  int nx, ny, bcx, bcy;
  double dn, dtan;
  float dnf, itanf, gammaf, epsf;   // single-precision copies (dn, 1/dtan, gamma, WENO eps)
  int stage;
  PhysParams P;
  const StepTimes* tc;  // the step's time constants (same storage as dtp)
};

// FP32-bulk cell update: FP64 accumulation; writes the next mirror.
struct UpdateArgs32 {
  double* W;           // FP64 state [W | Wx (| Wy)][nv][ny][nx]: W^n read and W^{n+1} written (stage 2)
  float* fx;           // x-face buffer (one FP64 block, then five FP32 blocks; see write_face32)
  float* fy;           // y-face buffer (2D)
  float* M;            // FP32 mirror: W^n / W* / W^{n+1} (hi, lo, Wx, Wy planes)
  int nx, ny, bcx, bcy;
  double idx, idy;
};

// launchers (defined in the .cu units)
cudaError_t launch_mirror(const double* S, float* M, int nx, int ny, int dim, cudaStream_t s);
// the mirror of rows [j0, j0 + nrows) only
cudaError_t launch_mirror_rows(const double* S, float* M, int nx, int ny, int dim, int j0, int nrows,
                               cudaStream_t s);
cudaError_t launch_faces32_1d(const FaceArgs32& a, int order, int recon, bool visc, cudaStream_t s);
cudaError_t launch_faces32_2d(const FaceArgs32& a, int dir, int order, int recon, bool visc, cudaStream_t s);
cudaError_t launch_update32(const UpdateArgs32& a, int dim, int stage, cudaStream_t s);
cudaError_t launch_faces_1d(const FaceArgs& a, int order, int recon, bool visc, cudaStream_t s);
cudaError_t launch_faces_2d(const FaceArgs& a, int dir, int order, int recon, bool visc, cudaStream_t s);
cudaError_t launch_update(const UpdateArgs& a, int dim, int stage, cudaStream_t s);
cudaError_t launch_wavespeed(const double* W, int nx, int ny, int dim, double gamma, double dx,
                             double dy, unsigned long long* out, cudaStream_t s);
cudaError_t launch_set_scalar(double* p, double v, cudaStream_t s);
cudaError_t launch_set_times(StepTimes* p, double dt, cudaStream_t s);
cudaError_t probe_fma(int fp64, int iters, double* flops, cudaStream_t s);
cudaError_t probe_time_coefs(const double* theta, int n, double dt, double* out, bool single);

// Test probe: the FP32-bulk sweeps' FP64 reciprocal of host x[0..n) into host out.
cudaError_t probe_rcp64(const double* x, int n, double* out);
cudaError_t probe_d2f(const double* x, int n, float* out);

}  // namespace gks
