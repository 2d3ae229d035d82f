// gks_update.cu -- cell updates of the two-stage MSMD step and the CFL reduction.
//
// Stage 1 (Eq. step-hyper-1 and the interface-value MSMD of Sec. 2.2):
//   W*   = W^n - [Phi]_x/dx - [Phi]_y/dy            Phi = dt/2 F + dt^2/8 F_t
//   W_x* = [Omega]_x/dx, W_y* = [Omega]_y/dy        Omega = W0 + dt/2 W_t + dt^2/8 W_tt
//   acc  = W^n - [Psi]_x/dx - [Psi]_y/dy            Psi = dt F + dt^2/6 F_t
//   accx = [Lambda]_x/dx, accy = [Lambda]_y/dy      Lambda = W0 + dt W_t + dt^2/6 W_tt
// Stage 2 (Eq. step-hyper-2):
//   W^{n+1}   = acc  - [dt^2/3 F_t*]_x/dx - [dt^2/3 F_t*]_y/dy
//   W_x^{n+1} = accx + [dt^2/3 W_tt*]_x/dx, W_y^{n+1} = accy + [dt^2/3 W_tt*]_y/dy
// [q]_x is the difference of face values across the cell (Gauss formula, Eq.
// Gausian-formula, for the slopes).
#include "gks_kernels.cuh"

namespace gks {

template <int DIM, int STAGE>
__global__ void __launch_bounds__(256) update_kernel(UpdateArgs a) {
  const int N = DIM + 2;
  const long ncell = (long)a.nx * a.ny;
  long c = (long)blockIdx.x * blockDim.x + threadIdx.x;
  if (c >= ncell) return;
  int j = (int)(c / a.nx), i = (int)(c - (long)j * a.nx);
  const long nfx = (long)a.ny * (a.nx + 1);
  const long fxl = (long)j * (a.nx + 1) + i;
  const long nfy = (long)(a.ny + 1) * a.nx;
  const long fyb = (long)j * a.nx + i;
  const long fyt = fyb + a.nx;
  double* Wo = a.Ws;
  double* Wxo = a.Ws + N * ncell;
  double* Wyo = a.Ws + 2 * N * ncell;
  double* accW = a.acc;
  double* accX = a.acc + N * ncell;
  double* accY = a.acc + 2 * N * ncell;
#pragma unroll
  for (int v = 0; v < N; ++v) {
    const long p = v * ncell + c;
    if (STAGE == 1) {
      const double* Phi = a.fx + (0L * N + v) * nfx;
      const double* Psi = a.fx + (1L * N + v) * nfx;
      const double* Om = a.fx + (2L * N + v) * nfx;
      const double* La = a.fx + (3L * N + v) * nfx;
      double ws = a.W[p] - (Phi[fxl + 1] - Phi[fxl]) * a.idx;
      double wa = a.W[p] - (Psi[fxl + 1] - Psi[fxl]) * a.idx;
      Wxo[p] = (Om[fxl + 1] - Om[fxl]) * a.idx;
      accX[p] = (La[fxl + 1] - La[fxl]) * a.idx;
      if (DIM == 2) {
        const double* PhiY = a.fy + (0L * N + v) * nfy;
        const double* PsiY = a.fy + (1L * N + v) * nfy;
        const double* OmY = a.fy + (2L * N + v) * nfy;
        const double* LaY = a.fy + (3L * N + v) * nfy;
        ws -= (PhiY[fyt] - PhiY[fyb]) * a.idy;
        wa -= (PsiY[fyt] - PsiY[fyb]) * a.idy;
        Wyo[p] = (OmY[fyt] - OmY[fyb]) * a.idy;
        accY[p] = (LaY[fyt] - LaY[fyb]) * a.idy;
      }
      Wo[p] = ws;
      accW[p] = wa;
    } else {
      const double* Ft = a.fx + (0L * N + v) * nfx;
      const double* Tt = a.fx + (1L * N + v) * nfx;
      double w = accW[p] - (Ft[fxl + 1] - Ft[fxl]) * a.idx;
      Wxo[p] = accX[p] + (Tt[fxl + 1] - Tt[fxl]) * a.idx;
      if (DIM == 2) {
        const double* FtY = a.fy + (0L * N + v) * nfy;
        const double* TtY = a.fy + (1L * N + v) * nfy;
        w -= (FtY[fyt] - FtY[fyb]) * a.idy;
        Wyo[p] = accY[p] + (TtY[fyt] - TtY[fyb]) * a.idy;
      }
      Wo[p] = w;
    }
  }
}

cudaError_t launch_update(const UpdateArgs& a, int dim, int stage, cudaStream_t s) {
  long ncell = (long)a.nx * a.ny;
  int threads = 256;
  unsigned blocks = (unsigned)((ncell + threads - 1) / threads);
  if (dim == 1) {
    if (stage == 1) update_kernel<1, 1><<<blocks, threads, 0, s>>>(a);
    else update_kernel<1, 2><<<blocks, threads, 0, s>>>(a);
  } else {
    if (stage == 1) update_kernel<2, 1><<<blocks, threads, 0, s>>>(a);
    else update_kernel<2, 2><<<blocks, threads, 0, s>>>(a);
  }
  return cudaGetLastError();
}

// max over cells of (|U| + c)/dx (+ (|V| + c)/dy): block reduction, then an atomic max on
// the bit pattern (valid ordering for non-negative doubles).  A non-finite or
// non-physical cell stores +inf.
template <int DIM>
__global__ void __launch_bounds__(256) wavespeed_kernel(const double* W, long ncell, double gamma,
                                                        double idx, double idy,
                                                        unsigned long long* out) {
  __shared__ double red[256];
  double m = 0.0;
  for (long c = (long)blockIdx.x * blockDim.x + threadIdx.x; c < ncell; c += (long)gridDim.x * blockDim.x) {
    double rho = W[c], U = W[ncell + c] / rho;
    double V = DIM == 2 ? W[2 * ncell + c] / rho : 0.0;
    double E = W[(DIM + 1) * ncell + c];
    double p = (gamma - 1.0) * (E - 0.5 * rho * (U * U + V * V));
    double s;
    if (!(rho > 0.0) || !(p > 0.0)) s = __longlong_as_double(0x7ff0000000000000LL);
    else {
      double cs = sqrt(gamma * p / rho);
      s = (fabs(U) + cs) * idx;
      if (DIM == 2) s += (fabs(V) + cs) * idy;
    }
    m = fmax(m, s);
  }
  red[threadIdx.x] = m;
  __syncthreads();
  for (int w = blockDim.x / 2; w > 0; w >>= 1) {
    if (threadIdx.x < w) red[threadIdx.x] = fmax(red[threadIdx.x], red[threadIdx.x + w]);
    __syncthreads();
  }
  if (threadIdx.x == 0) atomicMax(out, (unsigned long long)__double_as_longlong(red[0]));
}

cudaError_t launch_wavespeed(const double* W, int nx, int ny, int dim, double gamma, double dx,
                             double dy, unsigned long long* out, cudaStream_t s) {
  long ncell = (long)nx * ny;
  cudaError_t e = cudaMemsetAsync(out, 0, sizeof(unsigned long long), s);
  if (e != cudaSuccess) return e;
  int threads = 256;
  long want = (ncell + threads - 1) / threads;
  int blocks = (int)(want < 152 * 8 ? (want > 0 ? want : 1) : 152 * 8);
  if (dim == 1) wavespeed_kernel<1><<<blocks, threads, 0, s>>>(W, ncell, gamma, 1.0 / dx, 0.0, out);
  else wavespeed_kernel<2><<<blocks, threads, 0, s>>>(W, ncell, gamma, 1.0 / dx, 1.0 / dy, out);
  return cudaGetLastError();
}

__global__ void set_scalar_kernel(double* p, double v) { *p = v; }

__global__ void set_times_kernel(StepTimes* p, double dt) { *p = step_times(dt); }

cudaError_t launch_set_times(StepTimes* p, double dt, cudaStream_t s) {
  set_times_kernel<<<1, 1, 0, s>>>(p, dt);
  return cudaGetLastError();
}

cudaError_t launch_set_scalar(double* p, double v, cudaStream_t s) {
  set_scalar_kernel<<<1, 1, 0, s>>>(p, v);
  return cudaGetLastError();
}

}  // namespace gks
