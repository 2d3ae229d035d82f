// gks_static.cu -- one 1D two-stage step that allocates nothing.
//
// Some callers cannot call cudaMalloc: code running inside a memory pool they do not own,
// plug-ins whose host forbids device allocation after start-up, or real-time loops where
// an allocation (and the implicit synchronisation it may bring) is not allowed.  For them
// gks_step_1d_static runs the same face-sweep and update kernels as gks_step, with all its
// scratch in one file-scope device array sized for at most GKS_STATIC_MAX_NX cells.
// Every GPU that loads the library holds this array until the process exits.
#include <cuda_runtime.h>
#include <math.h>
#include <stdio.h>
#include <mutex>
#include <string>

#include "../../include/gks.h"
#include "gks_kernels.cuh"

namespace {

constexpr long NX_MAX = GKS_STATIC_MAX_NX;
// scratch layout (in doubles), 1D, 3 conservative variables:
//   stage state W*, W_x*       2 * 3 * NX_MAX
//   accumulators               2 * 3 * NX_MAX
//   result W, W_x              2 * 3 * NX_MAX
//   x-face buffer              4 * 3 * (NX_MAX + 1)
//   dt, status                 2 slots (status read as unsigned int)
constexpr long OFF_STAGE = 0;
constexpr long OFF_ACC = OFF_STAGE + 6 * NX_MAX;
constexpr long OFF_OUT = OFF_ACC + 6 * NX_MAX;
constexpr long OFF_FACES = OFF_OUT + 6 * NX_MAX;
constexpr long OFF_DT = OFF_FACES + 12 * (NX_MAX + 1);
constexpr long OFF_STATUS = OFF_DT + 1;
constexpr long SCRATCH_DOUBLES = OFF_STATUS + 1;

static __device__ __align__(256) double g_scratch[SCRATCH_DOUBLES];

constexpr int MAX_DEVICES = 64;
std::mutex g_mutex;
double* g_scratch_addr[MAX_DEVICES] = {nullptr};

thread_local std::string g_static_err;

int sfail(int code, const char* msg) {
  g_static_err = msg;
  return code;
}
int scuda(cudaError_t e, const char* where) {
  char buf[256];
  snprintf(buf, sizeof(buf), "%s: %s", where, cudaGetErrorString(e));
  g_static_err = buf;
  return GKS_ECUDA;
}

// Device address of the scratch array on the current device, looked up once per device.
int scratch_on_current_device(double** out) {
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return scuda(e, "cudaGetDevice");
  if (dev < 0 || dev >= MAX_DEVICES) return sfail(GKS_EINVAL, "device index out of range");
  std::lock_guard<std::mutex> lock(g_mutex);
  if (!g_scratch_addr[dev]) {
    void* p = nullptr;
    e = cudaGetSymbolAddress(&p, g_scratch);
    if (e != cudaSuccess) return scuda(e, "cudaGetSymbolAddress(scratch)");
    g_scratch_addr[dev] = static_cast<double*>(p);
  }
  *out = g_scratch_addr[dev];
  return GKS_OK;
}

}  // namespace

extern "C" int gks_step_1d_static(const double* W, const double* Wx, double* W_out, double* Wx_out,
                                  int nx, double gamma, double mu, double Pr, double x0, double x1,
                                  int bc, int order, int recon, double dt, void* stream) {
  g_static_err.clear();
  if (!W || !Wx || !W_out || !Wx_out) return sfail(GKS_EINVAL, "NULL state pointer");
  if (nx < 5) return sfail(GKS_EINVAL, "nx must be >= 5");
  if (nx > GKS_STATIC_MAX_NX) return sfail(GKS_EINVAL, "nx exceeds GKS_STATIC_MAX_NX (the size of the static scratch)");
  if (order != 6 && order != 8) return sfail(GKS_EINVAL, "order must be 6 or 8");
  if (recon != GKS_RECON_LINEAR && recon != GKS_RECON_WENOZ) return sfail(GKS_EINVAL, "recon must be 0 or 1");
  if (bc != GKS_BC_PERIODIC && bc != GKS_BC_TRANSMISSIVE && bc != GKS_BC_REFLECTING) return sfail(GKS_EINVAL, "bc must be 0, 1 or 2");
  if (!isfinite(gamma) || !isfinite(mu) || !isfinite(Pr) || !(gamma > 1.0) || !(mu >= 0.0) || !(Pr > 0.0))
    return sfail(GKS_EINVAL, "need finite gamma > 1, mu >= 0, Pr > 0");
  if (!isfinite(x0) || !isfinite(x1) || !(x1 > x0)) return sfail(GKS_EINVAL, "domain must be finite and non-empty");
  if (!(dt > 0.0) || !isfinite(dt)) return sfail(GKS_EINVAL, "dt must be finite and > 0");

  double* s = nullptr;
  int rc = scratch_on_current_device(&s);
  if (rc != GKS_OK) return rc;
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  const long L = 3L * nx;
  const double dx = (x1 - x0) / nx;
  unsigned int* status = reinterpret_cast<unsigned int*>(s + OFF_STATUS);
  double* dtp = s + OFF_DT;

  cudaError_t e = cudaMemsetAsync(status, 0, sizeof(unsigned int), st);
  if (e != cudaSuccess) return scuda(e, "status clear");
  e = gks::launch_set_scalar(dtp, dt, st);
  if (e != cudaSuccess) return scuda(e, "dt");

  gks::FaceArgs fa;
  fa.dtp = dtp; fa.status = status;
  fa.nx = nx; fa.ny = 1; fa.bcx = bc; fa.bcy = 0;
  fa.dn = dx; fa.dtan = 1.0;
  fa.P.gamma = gamma; fa.P.K = (3.0 - gamma) / (gamma - 1.0);
  fa.P.mu = mu; fa.P.Pr = Pr; fa.P.eps_tau = 0.01; fa.P.C_tau = 1.0; fa.P.weno_eps = 1e-6;
  gks::set_phys_floats(fa.P);
  fa.out = s + OFF_FACES;
  gks::UpdateArgs ua;
  ua.fx = s + OFF_FACES; ua.fy = nullptr; ua.acc = s + OFF_ACC;
  ua.nx = nx; ua.ny = 1; ua.idx = 1.0 / dx; ua.idy = 1.0;
  const bool visc = mu > 0.0;
  // stage 1 on the caller's state
  fa.stage = 1; fa.W = W; fa.Wn = Wx;
  e = gks::launch_faces_1d(fa, order, recon, visc, st);
  if (e != cudaSuccess) return scuda(e, "face sweep 1");
  ua.W = W; ua.Ws = s + OFF_STAGE;
  e = gks::launch_update(ua, 1, 1, st);
  if (e != cudaSuccess) return scuda(e, "update 1");
  // stage 2 on W*
  fa.stage = 2; fa.W = s + OFF_STAGE; fa.Wn = s + OFF_STAGE + L;
  e = gks::launch_faces_1d(fa, order, recon, visc, st);
  if (e != cudaSuccess) return scuda(e, "face sweep 2");
  ua.W = s + OFF_STAGE; ua.Ws = s + OFF_OUT;
  e = gks::launch_update(ua, 1, 2, st);
  if (e != cudaSuccess) return scuda(e, "update 2");
  e = cudaMemcpyAsync(W_out, s + OFF_OUT, L * sizeof(double), cudaMemcpyDeviceToDevice, st);
  if (e == cudaSuccess) e = cudaMemcpyAsync(Wx_out, s + OFF_OUT + L, L * sizeof(double), cudaMemcpyDeviceToDevice, st);
  if (e != cudaSuccess) return scuda(e, "result copy");
  unsigned int hs = 0;
  e = cudaMemcpyAsync(&hs, status, sizeof(hs), cudaMemcpyDeviceToHost, st);
  if (e == cudaSuccess) e = cudaStreamSynchronize(st);
  if (e != cudaSuccess) return scuda(e, "synchronise");
  if (hs & gks::ST_NONPHYSICAL) return sfail(GKS_ENONPHYSICAL, "non-physical interface state (rho <= 0 or p <= 0)");
  return GKS_OK;
}

extern "C" const char* gks_static_last_error(void) { return g_static_err.c_str(); }
