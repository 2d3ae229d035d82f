// gks_api.cu -- C ABI (include/gks.h): context, buffers, the two-stage step as a CUDA graph.
#include <cuda_runtime.h>
#include <stdio.h>
#include <stdlib.h>
#include <string.h>
#include <cmath>
#include <new>
#include <string>

#include "../../include/gks.h"
#include "gks_kernels.cuh"

namespace {

thread_local std::string g_err;

int fail(int code, const char* fmt, const char* detail = nullptr) {
  char buf[512];
  snprintf(buf, sizeof(buf), fmt, detail ? detail : "");
  g_err = buf;
  return code;
}
int cuda_fail(cudaError_t e, const char* where) {
  char buf[512];
  snprintf(buf, sizeof(buf), "%s: %s", where, cudaGetErrorString(e));
  g_err = buf;
  return e == cudaErrorMemoryAllocation ? GKS_ENOMEM : GKS_ECUDA;
}

}  // namespace

struct gks_ctx {
  int nx = 0, ny = 0, dim = 1, nv = 3, order = 6, recon = 0;
  gks_opts o;
  gks::PhysParams P;
  double dx = 1, dy = 1;
  long ncell = 0;
  cudaStream_t stream = nullptr;
  bool own_stream = false;
  // device buffers
  double* state = nullptr;   // [W | Wx | Wy] each nv*ncell
  double* stage = nullptr;   // W*, Wx*, Wy*
  double* acc = nullptr;     // accumulators
  double* fx = nullptr;      // x-face buffer [4][nv][ny][nx+1]
  double* fy = nullptr;      // y-face buffer [4][nv][ny+1][nx]
  double* d_dt = nullptr;
  float* mirror = nullptr;   // FP32-bulk: [hi | lo | Wx | Wy] floats
  unsigned int* d_status = nullptr;
  unsigned long long* d_ws = nullptr;
  double last_dt = -1.0;
  cudaGraph_t graph = nullptr;
  cudaGraphExec_t exec = nullptr;
};

namespace {

long state_len(const gks_ctx* c) { return (long)c->nv * c->ncell; }

// Enqueue the two-stage step (no dt update) on the context stream.  When ev is given,
// launch slot k is bracketed by events ev[2k], ev[2k+1].
int enqueue_step(gks_ctx* c, cudaEvent_t* ev = nullptr) {
  int slot = 0;
  auto mark = [&](bool begin) {
    if (ev) cudaEventRecord(ev[2 * slot + (begin ? 0 : 1)], c->stream);
    if (!begin) ++slot;
  };
  cudaError_t e;
  if (c->o.precision == GKS_PREC_FP32_BULK) {
    const long L = state_len(c);
    gks::FaceArgs32 fa;
    fa.dtp = c->d_dt; fa.status = c->d_status;
    fa.tc = reinterpret_cast<const gks::StepTimes*>(c->d_dt);
    fa.nx = c->nx; fa.ny = c->ny; fa.bcx = c->o.bc_x; fa.bcy = c->o.bc_y;
    fa.P = c->P;
    fa.M = c->mirror;
    fa.W = c->state;
    fa.dnf = (float)c->dx; fa.gammaf = (float)c->P.gamma; fa.epsf = (float)c->P.weno_eps;
    const bool visc = c->P.mu > 0.0 || c->P.tau_mode == 1;
    gks::UpdateArgs32 ua;
    ua.fx = reinterpret_cast<float*>(c->fx); ua.fy = reinterpret_cast<float*>(c->fy);
    ua.W = c->state; ua.M = c->mirror;
    ua.nx = c->nx; ua.ny = c->ny; ua.bcx = c->o.bc_x; ua.bcy = c->o.bc_y;
    ua.idx = 1.0 / c->dx; ua.idy = 1.0 / c->dy;
    for (int stage = 1; stage <= 2; ++stage) {
      fa.stage = stage;
      fa.Mn = c->mirror + 2 * L; fa.out = c->fx; fa.dn = c->dx; fa.dtan = c->dy;
      fa.dnf = (float)c->dx; fa.itanf = (float)(1.0 / c->dy);
      mark(true);
      if (c->dim == 1) e = gks::launch_faces32_1d(fa, c->order, c->recon, visc, c->stream);
      else e = gks::launch_faces32_2d(fa, 0, c->order, c->recon, visc, c->stream);
      mark(false);
      if (e != cudaSuccess) return cuda_fail(e, "x-face sweep (fp32)");
      if (c->dim == 2) {
        fa.Mn = c->mirror + 3 * L; fa.out = c->fy; fa.dn = c->dy; fa.dtan = c->dx;
        fa.dnf = (float)c->dy; fa.itanf = (float)(1.0 / c->dx);
        mark(true);
        e = gks::launch_faces32_2d(fa, 1, c->order, c->recon, visc, c->stream);
        mark(false);
        if (e != cudaSuccess) return cuda_fail(e, "y-face sweep (fp32)");
      }
      mark(true);
      e = gks::launch_update32(ua, c->dim, stage, c->stream);
      mark(false);
      if (e != cudaSuccess) return cuda_fail(e, "cell update (fp32)");
    }
    return GKS_OK;
  }
  gks::FaceArgs fa;
  fa.dtp = c->d_dt; fa.status = c->d_status;
  fa.nx = c->nx; fa.ny = c->ny; fa.bcx = c->o.bc_x; fa.bcy = c->o.bc_y;
  fa.P = c->P;
  const bool visc = c->P.mu > 0.0 || c->P.tau_mode == 1;
  const long L = state_len(c);
  gks::UpdateArgs ua;
  ua.fx = c->fx; ua.fy = c->fy; ua.acc = c->acc;
  ua.nx = c->nx; ua.ny = c->ny; ua.idx = 1.0 / c->dx; ua.idy = 1.0 / c->dy;
  for (int stage = 1; stage <= 2; ++stage) {
    const double* W = stage == 1 ? c->state : c->stage;
    fa.stage = stage;
    fa.W = W;
    // x faces
    fa.Wn = W + L; fa.out = c->fx; fa.dn = c->dx; fa.dtan = c->dy;
    mark(true);
    if (c->dim == 1) e = gks::launch_faces_1d(fa, c->order, c->recon, visc, c->stream);
    else e = gks::launch_faces_2d(fa, 0, c->order, c->recon, visc, c->stream);
    mark(false);
    if (e != cudaSuccess) return cuda_fail(e, "x-face sweep");
    if (c->dim == 2) {
      fa.Wn = W + 2 * L; fa.out = c->fy; fa.dn = c->dy; fa.dtan = c->dx;
      mark(true);
      e = gks::launch_faces_2d(fa, 1, c->order, c->recon, visc, c->stream);
      mark(false);
      if (e != cudaSuccess) return cuda_fail(e, "y-face sweep");
    }
    ua.W = W;
    ua.Ws = stage == 1 ? c->stage : c->state;
    mark(true);
    e = gks::launch_update(ua, c->dim, stage, c->stream);
    mark(false);
    if (e != cudaSuccess) return cuda_fail(e, "cell update");
  }
  return GKS_OK;
}

// FP32-bulk: rebuild the float mirror after the FP64 state was replaced.
int refresh_mirror(gks_ctx* c) {
  if (c->o.precision != GKS_PREC_FP32_BULK) return GKS_OK;
  cudaError_t e = gks::launch_mirror(c->state, c->mirror, c->nx, c->ny, c->dim, c->stream);
  if (e != cudaSuccess) return cuda_fail(e, "mirror");
  return GKS_OK;
}

int check_status(gks_ctx* c) {
  unsigned int st = 0;
  cudaError_t e = cudaMemcpyAsync(&st, c->d_status, sizeof(st), cudaMemcpyDeviceToHost, c->stream);
  if (e == cudaSuccess) e = cudaStreamSynchronize(c->stream);
  if (e != cudaSuccess) return cuda_fail(e, "status read");
  if (st & gks::ST_NONPHYSICAL) return fail(GKS_ENONPHYSICAL, "non-physical interface state (rho <= 0 or p <= 0)%s");
  return GKS_OK;
}

}  // namespace

extern "C" {

void gks_default_opts(gks_opts* o) {
  if (!o) return;
  memset(o, 0, sizeof(*o));
  o->x0 = 0; o->x1 = 1; o->y0 = 0; o->y1 = 1;
  o->bc_x = GKS_BC_PERIODIC; o->bc_y = GKS_BC_PERIODIC;
  o->precision = GKS_PREC_FP64;
  o->weno_eps = 1e-12;
  o->eps_tau = 0.01; o->C_tau = 1.0;
  o->use_graph = 1;
  o->tau_mode = 0;
  o->stream = nullptr;
}

const char* gks_last_error(void) { return g_err.c_str(); }

gks_ctx* gks_create(int nx, int ny, double gamma, double mu, double Pr, int order, int recon,
                    const gks_opts* opts) {
  g_err.clear();
  if (nx < 5 || ny < 1 || (ny > 1 && ny < 5)) { fail(GKS_EINVAL, "grid must have nx >= 5 and ny == 1 or ny >= 5%s"); return nullptr; }
  if ((long)nx * ny > (1L << 31)) { fail(GKS_EINVAL, "grid too large%s"); return nullptr; }
  if (order != 6 && order != 8) { fail(GKS_EINVAL, "order must be 6 or 8%s"); return nullptr; }
  if (recon != GKS_RECON_LINEAR && recon != GKS_RECON_WENOZ) { fail(GKS_EINVAL, "recon must be 0 (linear) or 1 (WENO-Z)%s"); return nullptr; }
  if (!(gamma > 1.0) || !std::isfinite(gamma)) { fail(GKS_EINVAL, "gamma must be > 1%s"); return nullptr; }
  if (!(mu >= 0.0) || !std::isfinite(mu)) { fail(GKS_EINVAL, "mu must be >= 0%s"); return nullptr; }
  if (!(Pr > 0.0) || !std::isfinite(Pr)) { fail(GKS_EINVAL, "Pr must be > 0%s"); return nullptr; }
  gks_opts o;
  if (opts) o = *opts; else gks_default_opts(&o);
  if (!(o.x1 > o.x0) || (ny > 1 && !(o.y1 > o.y0))) { fail(GKS_EINVAL, "empty domain%s"); return nullptr; }
  if (o.bc_x < 0 || o.bc_x > 2 || o.bc_y < 0 || o.bc_y > 2) { fail(GKS_EINVAL, "bc must be 0, 1 or 2%s"); return nullptr; }
  if (o.precision != GKS_PREC_FP64 && o.precision != GKS_PREC_FP32_BULK) { fail(GKS_EINVAL, "unsupported precision%s"); return nullptr; }
  if (!(o.weno_eps > 0.0) || !(o.eps_tau > 0.0) || !(o.C_tau >= 0.0)) { fail(GKS_EINVAL, "weno_eps, eps_tau must be > 0 and C_tau >= 0%s"); return nullptr; }
  if (o.tau_mode != 0 && o.tau_mode != 1) { fail(GKS_EINVAL, "tau_mode must be 0 or 1%s"); return nullptr; }

  gks_ctx* c = new (std::nothrow) gks_ctx();
  if (!c) { fail(GKS_ENOMEM, "host allocation failed%s"); return nullptr; }
  c->nx = nx; c->ny = ny; c->dim = ny > 1 ? 2 : 1; c->nv = c->dim + 2;
  c->order = order; c->recon = recon; c->o = o;
  c->dx = (o.x1 - o.x0) / nx;
  c->dy = c->dim == 2 ? (o.y1 - o.y0) / ny : 1.0;
  c->ncell = (long)nx * ny;
  c->P.gamma = gamma;
  c->P.K = c->dim == 1 ? (3.0 - gamma) / (gamma - 1.0) : (4.0 - 2.0 * gamma) / (gamma - 1.0);
  c->P.mu = mu; c->P.Pr = Pr;
  c->P.eps_tau = o.eps_tau; c->P.C_tau = o.C_tau; c->P.weno_eps = o.weno_eps;
  c->P.tau_mode = o.tau_mode;
  gks::set_phys_floats(c->P);

  cudaError_t e;
  if (o.stream) c->stream = (cudaStream_t)o.stream;
  else {
    e = cudaStreamCreateWithFlags(&c->stream, cudaStreamNonBlocking);
    if (e != cudaSuccess) { cuda_fail(e, "stream create"); delete c; return nullptr; }
    c->own_stream = true;
  }
  const long L = state_len(c);
  const int nsets = c->dim + 1;   // W, Wx (, Wy)
  size_t fxn = (size_t)4 * c->nv * ny * (nx + 1);
  size_t fyn = c->dim == 2 ? (size_t)4 * c->nv * (ny + 1) * nx : 0;
  // the FP64 form keeps W* and the MSMD accumulators; the FP32-bulk form folds both stages
  // into the face data and keeps only the state and its float mirror
  const size_t nstage = o.precision == GKS_PREC_FP64 ? (size_t)nsets * L : 0;
  struct { double** p; size_t n; } bufs[] = {
      {&c->state, (size_t)nsets * L}, {&c->stage, nstage}, {&c->acc, nstage},
      {&c->fx, fxn}, {&c->fy, fyn}, {&c->d_dt, (size_t)gks::STEP_TIMES_DOUBLES}};
  for (auto& b : bufs) {
    if (b.n == 0) continue;
    e = cudaMalloc((void**)b.p, b.n * sizeof(double));
    if (e != cudaSuccess) { cuda_fail(e, "device allocation"); gks_destroy(c); return nullptr; }
  }
  if (o.precision == GKS_PREC_FP32_BULK) {
    e = cudaMalloc((void**)&c->mirror, (size_t)(c->dim + 2) * L * sizeof(float));
    if (e != cudaSuccess) { cuda_fail(e, "device allocation"); gks_destroy(c); return nullptr; }
  }
  e = cudaMalloc((void**)&c->d_status, sizeof(unsigned int));
  if (e == cudaSuccess) e = cudaMalloc((void**)&c->d_ws, sizeof(unsigned long long));
  if (e == cudaSuccess) e = cudaMemsetAsync(c->d_status, 0, sizeof(unsigned int), c->stream);
  if (e == cudaSuccess) e = cudaMemsetAsync(c->state, 0, (size_t)nsets * L * sizeof(double), c->stream);
  if (e == cudaSuccess) e = cudaStreamSynchronize(c->stream);
  if (e != cudaSuccess) { cuda_fail(e, "device allocation"); gks_destroy(c); return nullptr; }
  return c;
}

int gks_set_state(gks_ctx* c, const double* W, const double* Wx, const double* Wy) {
  if (!c || !W || !Wx || (c->dim == 2 && !Wy)) return fail(GKS_EINVAL, "NULL argument%s");
  const long L = state_len(c);
  const double* src[3] = {W, Wx, Wy};
  for (int k = 0; k <= c->dim; ++k) {
    cudaError_t e = cudaMemcpyAsync(c->state + k * L, src[k], L * sizeof(double), cudaMemcpyHostToDevice, c->stream);
    if (e != cudaSuccess) return cuda_fail(e, "set_state copy");
  }
  int rc = refresh_mirror(c);
  if (rc != GKS_OK) return rc;
  cudaError_t e = cudaStreamSynchronize(c->stream);
  if (e != cudaSuccess) return cuda_fail(e, "set_state");
  return GKS_OK;
}

int gks_set_state_device(gks_ctx* c, const double* W, const double* Wx, const double* Wy) {
  if (!c || !W || !Wx || (c->dim == 2 && !Wy)) return fail(GKS_EINVAL, "NULL argument%s");
  const long L = state_len(c);
  const double* src[3] = {W, Wx, Wy};
  for (int k = 0; k <= c->dim; ++k) {
    cudaError_t e = cudaMemcpyAsync(c->state + k * L, src[k], L * sizeof(double), cudaMemcpyDeviceToDevice, c->stream);
    if (e != cudaSuccess) return cuda_fail(e, "set_state_device copy");
  }
  return refresh_mirror(c);
}

int gks_get_state(gks_ctx* c, double* W, double* Wx, double* Wy) {
  if (!c || !W || !Wx || (c->dim == 2 && !Wy)) return fail(GKS_EINVAL, "NULL argument%s");
  const long L = state_len(c);
  double* dst[3] = {W, Wx, Wy};
  for (int k = 0; k <= c->dim; ++k) {
    cudaError_t e = cudaMemcpyAsync(dst[k], c->state + k * L, L * sizeof(double), cudaMemcpyDeviceToHost, c->stream);
    if (e != cudaSuccess) return cuda_fail(e, "get_state copy");
  }
  return check_status(c);
}

int gks_get_state_device(gks_ctx* c, double* W, double* Wx, double* Wy) {
  if (!c || !W || !Wx || (c->dim == 2 && !Wy)) return fail(GKS_EINVAL, "NULL argument%s");
  const long L = state_len(c);
  double* dst[3] = {W, Wx, Wy};
  for (int k = 0; k <= c->dim; ++k) {
    cudaError_t e = cudaMemcpyAsync(dst[k], c->state + k * L, L * sizeof(double), cudaMemcpyDeviceToDevice, c->stream);
    if (e != cudaSuccess) return cuda_fail(e, "get_state_device copy");
  }
  return check_status(c);
}

int gks_steps(gks_ctx* c, double dt, int nsteps) {
  if (!c) return fail(GKS_EINVAL, "NULL context%s");
  if (!(dt > 0.0) || !std::isfinite(dt)) return fail(GKS_EINVAL, "dt must be finite and > 0%s");
  if (nsteps < 0) return fail(GKS_EINVAL, "nsteps must be >= 0%s");
  if (nsteps == 0) return GKS_OK;
  cudaError_t e;
  if (dt != c->last_dt) {
    e = gks::launch_set_times(reinterpret_cast<gks::StepTimes*>(c->d_dt), dt, c->stream);
    if (e != cudaSuccess) return cuda_fail(e, "dt update");
    c->last_dt = dt;
  }
  if (!c->o.use_graph) {
    for (int k = 0; k < nsteps; ++k) {
      int rc = enqueue_step(c);
      if (rc != GKS_OK) return rc;
    }
    return GKS_OK;
  }
  if (!c->exec) {
    e = cudaStreamBeginCapture(c->stream, cudaStreamCaptureModeThreadLocal);
    if (e != cudaSuccess) return cuda_fail(e, "graph capture begin");
    int rc = enqueue_step(c);
    cudaGraph_t g = nullptr;
    e = cudaStreamEndCapture(c->stream, &g);
    if (rc != GKS_OK) { if (g) cudaGraphDestroy(g); return rc; }
    if (e != cudaSuccess) return cuda_fail(e, "graph capture end");
    e = cudaGraphInstantiate(&c->exec, g, 0);
    if (e != cudaSuccess) { cudaGraphDestroy(g); return cuda_fail(e, "graph instantiate"); }
    c->graph = g;
  }
  for (int k = 0; k < nsteps; ++k) {
    e = cudaGraphLaunch(c->exec, c->stream);
    if (e != cudaSuccess) return cuda_fail(e, "graph launch");
  }
  return GKS_OK;
}

int gks_step(gks_ctx* c, double dt) { return gks_steps(c, dt, 1); }

int gks_steps_timed(gks_ctx* c, double dt, int nsteps, double* kernel_ms) {
  if (!c || !kernel_ms) return fail(GKS_EINVAL, "NULL argument%s");
  if (!(dt > 0.0) || !std::isfinite(dt)) return fail(GKS_EINVAL, "dt must be finite and > 0%s");
  if (nsteps < 0) return fail(GKS_EINVAL, "nsteps must be >= 0%s");
  const int nl = gks_launches_per_step(c);
  for (int k = 0; k < nl; ++k) kernel_ms[k] = 0.0;
  cudaError_t e;
  if (dt != c->last_dt) {
    e = gks::launch_set_times(reinterpret_cast<gks::StepTimes*>(c->d_dt), dt, c->stream);
    if (e != cudaSuccess) return cuda_fail(e, "dt update");
    c->last_dt = dt;
  }
  cudaEvent_t ev[12];
  for (int k = 0; k < 2 * nl; ++k) cudaEventCreate(&ev[k]);
  int rc = GKS_OK;
  for (int st = 0; st < nsteps && rc == GKS_OK; ++st) {
    rc = enqueue_step(c, ev);
    if (rc != GKS_OK) break;
    e = cudaEventSynchronize(ev[2 * nl - 1]);
    if (e != cudaSuccess) { rc = cuda_fail(e, "timed step"); break; }
    for (int k = 0; k < nl; ++k) {
      float ms = 0.f;
      cudaEventElapsedTime(&ms, ev[2 * k], ev[2 * k + 1]);
      kernel_ms[k] += ms;
    }
  }
  for (int k = 0; k < 2 * nl; ++k) cudaEventDestroy(ev[k]);
  return rc;
}

int gks_probe_alu_peak(int fp64, double* flops_per_s) {
  if (!flops_per_s) return fail(GKS_EINVAL, "NULL argument%s");
  cudaError_t e = gks::probe_fma(fp64, 1 << 14, flops_per_s, nullptr);
  if (e != cudaSuccess) return cuda_fail(e, "alu probe");
  return GKS_OK;
}

int gks_max_wavespeed(gks_ctx* c, double* out) {
  if (!c || !out) return fail(GKS_EINVAL, "NULL argument%s");
  cudaError_t e = gks::launch_wavespeed(c->state, c->nx, c->ny, c->dim, c->P.gamma, c->dx, c->dy, c->d_ws, c->stream);
  if (e != cudaSuccess) return cuda_fail(e, "wavespeed");
  unsigned long long bits = 0;
  e = cudaMemcpyAsync(&bits, c->d_ws, sizeof(bits), cudaMemcpyDeviceToHost, c->stream);
  if (e == cudaSuccess) e = cudaStreamSynchronize(c->stream);
  if (e != cudaSuccess) return cuda_fail(e, "wavespeed read");
  double v;
  memcpy(&v, &bits, sizeof(v));
  *out = v;
  if (!std::isfinite(v)) return fail(GKS_ENONPHYSICAL, "non-physical cell state (rho <= 0 or p <= 0)%s");
  return check_status(c);
}

int gks_sync(gks_ctx* c) {
  if (!c) return fail(GKS_EINVAL, "NULL context%s");
  return check_status(c);
}

int gks_state_device_ptrs(gks_ctx* c, double** W, double** Wx, double** Wy) {
  if (!c) return fail(GKS_EINVAL, "NULL context%s");
  const long L = state_len(c);
  if (W) *W = c->state;
  if (Wx) *Wx = c->state + L;
  if (Wy) *Wy = c->dim == 2 ? c->state + 2 * L : nullptr;
  return GKS_OK;
}

int gks_launches_per_step(gks_ctx* c) {
  if (!c) return fail(GKS_EINVAL, "NULL context%s");
  return c->dim == 2 ? 6 : 4;
}

void gks_destroy(gks_ctx* c) {
  if (!c) return;
  if (c->stream) cudaStreamSynchronize(c->stream);
  if (c->exec) cudaGraphExecDestroy(c->exec);
  if (c->graph) cudaGraphDestroy(c->graph);
  double* bufs[] = {c->state, c->stage, c->acc, c->fx, c->fy, c->d_dt};
  for (double* b : bufs) if (b) cudaFree(b);
  if (c->d_status) cudaFree(c->d_status);
  if (c->mirror) cudaFree(c->mirror);
  if (c->d_ws) cudaFree(c->d_ws);
  if (c->own_stream && c->stream) cudaStreamDestroy(c->stream);
  delete c;
}

}  // extern "C"
