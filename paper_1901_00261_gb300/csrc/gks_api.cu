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
  // FP32-bulk: the float mirror holds a pipeline slot's state, not `state` (rebuilt before the
  // next step of the context's own state)
  bool mirror_foreign = false;
  // pipelined host-to-host steps (gks_step_host_async): three state slots and three streams
  // of its own (copy-in, step, copy-out; created together so that they do not share a
  // hardware queue with one another, where they would run in submission order);
  // ev_in / ev_done / ev_out mark a slot's copy-in, step and copy-out.  pipe_pending: a
  // pipelined step may still be running, which the context stream joins (ev_done[pipe_last])
  // before its own next use of the shared buffers.
  double* slots = nullptr;
  cudaStream_t s_in = nullptr, s_comp = nullptr, s_out = nullptr;
  cudaEvent_t ev_in[3] = {}, ev_done[3] = {}, ev_out[3] = {}, ev_ctx = nullptr;
  long pipe_calls = 0;
  int pipe_last = 0;
  bool pipe_pending = false;
};

namespace {

long state_len(const gks_ctx* c) { return (long)c->nv * c->ncell; }

// Enqueue the two-stage step (no dt update) on the context stream.  When ev is given,
// launch slot k is bracketed by events ev[2k], ev[2k+1].
// state: the state to advance (default: the context's own).
int enqueue_step(gks_ctx* c, cudaEvent_t* ev = nullptr, double* state = nullptr) {
  double* const S = state ? state : c->state;
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
    fa.W = S;
    fa.dnf = (float)c->dx; fa.gammaf = (float)c->P.gamma; fa.epsf = (float)c->P.weno_eps;
    const bool visc = c->P.mu > 0.0 || c->P.tau_mode == 1;
    gks::UpdateArgs32 ua;
    ua.fx = reinterpret_cast<float*>(c->fx); ua.fy = reinterpret_cast<float*>(c->fy);
    ua.W = S; ua.M = c->mirror;
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
  for (int k = 0; k < 4; ++k) { fa.wallT[k] = c->o.wall_T[k]; fa.wallU[k] = c->o.wall_u[k]; }
  const bool visc = c->P.mu > 0.0 || c->P.tau_mode == 1;
  const long L = state_len(c);
  gks::UpdateArgs ua;
  ua.fx = c->fx; ua.fy = c->fy; ua.acc = c->acc;
  ua.nx = c->nx; ua.ny = c->ny; ua.idx = 1.0 / c->dx; ua.idy = 1.0 / c->dy;
  for (int stage = 1; stage <= 2; ++stage) {
    const double* W = stage == 1 ? S : c->stage;
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
    ua.Ws = stage == 1 ? c->stage : S;
    mark(true);
    e = gks::launch_update(ua, c->dim, stage, c->stream);
    mark(false);
    if (e != cudaSuccess) return cuda_fail(e, "cell update");
  }
  return GKS_OK;
}

// FP32-bulk: rebuild the float mirror after the FP64 state was replaced (state: a pipeline
// slot instead of the context's own state).
int refresh_mirror(gks_ctx* c, double* state = nullptr) {
  if (c->o.precision != GKS_PREC_FP32_BULK) return GKS_OK;
  cudaError_t e = gks::launch_mirror(state ? state : c->state, c->mirror, c->nx, c->ny, c->dim, c->stream);
  if (e != cudaSuccess) return cuda_fail(e, "mirror");
  c->mirror_foreign = state != nullptr;
  return GKS_OK;
}

// Before a step of the context's own state: the mirror must be that state's.
int own_mirror(gks_ctx* c) { return c->mirror_foreign ? refresh_mirror(c) : GKS_OK; }

// Order the context stream after the last pipelined step (they share the mirror, the face
// buffers and the step constants).
int join_pipeline(gks_ctx* c) {
  if (!c->pipe_pending) return GKS_OK;
  cudaError_t e = cudaStreamWaitEvent(c->stream, c->ev_done[c->pipe_last], 0);
  if (e != cudaSuccess) return cuda_fail(e, "pipeline join");
  c->pipe_pending = false;
  return GKS_OK;
}

int check_status(gks_ctx* c) {
  int jrc = join_pipeline(c);
  if (jrc != GKS_OK) return jrc;
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
  o->weno_eps = 1e-6;
  o->eps_tau = 0.01; o->C_tau = 1.0;
  o->use_graph = 1;
  o->tau_mode = 0;
  o->tan_mode = 0;
  o->stream = nullptr;
  for (int k = 0; k < 4; ++k) { o->wall_T[k] = 1.0; o->wall_u[k] = 0.0; }
  o->coef_mode = 0;
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
  if (o.bc_x < 0 || o.bc_x > 3 || o.bc_y < 0 || o.bc_y > 3) { fail(GKS_EINVAL, "bc must be 0, 1, 2 or 3%s"); return nullptr; }
  if (o.bc_x == GKS_BC_ISOTHERMAL || (ny > 1 && o.bc_y == GKS_BC_ISOTHERMAL)) {
    if (o.precision != GKS_PREC_FP64) { fail(GKS_EINVAL, "isothermal walls run in the FP64 form only%s"); return nullptr; }
    for (int k = 0; k < 4; ++k)
      if (!(o.wall_T[k] > 0.0) || !std::isfinite(o.wall_T[k]) || !std::isfinite(o.wall_u[k])) {
        fail(GKS_EINVAL, "wall_T must be finite and > 0, wall_u finite%s"); return nullptr;
      }
    // the mirror image of a moving wall moves the other way: a corner of a moving isothermal
    // wall and a reflecting one has no consistent ghost
    if (ny > 1 && ((o.bc_x == GKS_BC_REFLECTING && (o.wall_u[2] != 0.0 || o.wall_u[3] != 0.0)) ||
                   (o.bc_y == GKS_BC_REFLECTING && (o.wall_u[0] != 0.0 || o.wall_u[1] != 0.0)))) {
      fail(GKS_EINVAL, "a moving isothermal wall cannot meet a reflecting wall%s"); return nullptr;
    }
  }
  if (o.precision != GKS_PREC_FP64 && o.precision != GKS_PREC_FP32_BULK) { fail(GKS_EINVAL, "unsupported precision%s"); return nullptr; }
  if (!(o.weno_eps > 0.0) || !(o.eps_tau > 0.0) || !(o.C_tau >= 0.0)) { fail(GKS_EINVAL, "weno_eps, eps_tau must be > 0 and C_tau >= 0%s"); return nullptr; }
  if (o.tau_mode != 0 && o.tau_mode != 1) { fail(GKS_EINVAL, "tau_mode must be 0 or 1%s"); return nullptr; }
  if (o.tan_mode != 0 && o.tan_mode != 1) { fail(GKS_EINVAL, "tan_mode must be 0 or 1%s"); return nullptr; }
  if (o.coef_mode != 0 && o.coef_mode != 1) { fail(GKS_EINVAL, "coef_mode must be 0 or 1%s"); return nullptr; }
  if (o.coef_mode == 1 && (o.precision != GKS_PREC_FP64 || mu > 0.0 || o.tau_mode != 0 || o.tan_mode != 0)) {
    fail(GKS_EINVAL, "coef_mode 1 needs the FP64 form, mu = 0, tau_mode 0 and tan_mode 0%s"); return nullptr;
  }

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
  c->P.tan_mode = o.tan_mode;
  c->P.coef_mode = o.coef_mode;
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
  if (int jrc = join_pipeline(c)) return jrc;
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
  if (int jrc = join_pipeline(c)) return jrc;
  const long L = state_len(c);
  const double* src[3] = {W, Wx, Wy};
  for (int k = 0; k <= c->dim; ++k) {
    cudaError_t e = cudaMemcpyAsync(c->state + k * L, src[k], L * sizeof(double), cudaMemcpyDeviceToDevice, c->stream);
    if (e != cudaSuccess) return cuda_fail(e, "set_state_device copy");
  }
  return refresh_mirror(c);
}

namespace {
// One 2D copy of rows [j0, j0 + nrows) of every state plane (W, Wx, Wy; nvar planes each)
// between the state and a packed buffer [dim + 1][nvar][nrows][nx].
int copy_rows(gks_ctx* c, int j0, int nrows, double* buf, bool to_state, const char* what) {
  if (!c || !buf) return fail(GKS_EINVAL, "NULL argument%s");
  if (c->dim != 2) return fail(GKS_EINVAL, "rows exist in 2D only%s");
  if (j0 < 0 || nrows < 1 || (long)j0 + nrows > c->ny) return fail(GKS_EINVAL, "rows outside the grid%s");
  if (int jrc = join_pipeline(c)) return jrc;
  const size_t plane = (size_t)c->ny * c->nx * sizeof(double);
  const size_t width = (size_t)nrows * c->nx * sizeof(double);
  const size_t nplanes = (size_t)(c->dim + 1) * c->nv;
  double* rows = c->state + (size_t)j0 * c->nx;
  cudaError_t e = to_state
      ? cudaMemcpy2DAsync(rows, plane, buf, width, width, nplanes, cudaMemcpyDeviceToDevice, c->stream)
      : cudaMemcpy2DAsync(buf, width, rows, plane, width, nplanes, cudaMemcpyDeviceToDevice, c->stream);
  if (e != cudaSuccess) return cuda_fail(e, what);
  if (!to_state || c->o.precision != GKS_PREC_FP32_BULK) return GKS_OK;
  // the float mirror of the replaced rows (all of it if it holds a pipeline slot's state)
  if (c->mirror_foreign) return refresh_mirror(c);
  e = gks::launch_mirror_rows(c->state, c->mirror, c->nx, c->ny, c->dim, j0, nrows, c->stream);
  if (e != cudaSuccess) return cuda_fail(e, "mirror");
  return GKS_OK;
}
}  // namespace

int gks_get_rows_device(gks_ctx* c, int j0, int nrows, double* buf) {
  return copy_rows(c, j0, nrows, buf, false, "get_rows_device copy");
}

int gks_set_rows_device(gks_ctx* c, int j0, int nrows, const double* buf) {
  return copy_rows(c, j0, nrows, const_cast<double*>(buf), true, "set_rows_device copy");
}

int gks_get_state(gks_ctx* c, double* W, double* Wx, double* Wy) {
  if (!c || !W || !Wx || (c->dim == 2 && !Wy)) return fail(GKS_EINVAL, "NULL argument%s");
  if (int jrc = join_pipeline(c)) return jrc;
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
  if (int jrc = join_pipeline(c)) return jrc;
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
  if (int jrc = join_pipeline(c)) return jrc;
  int mrc = own_mirror(c);
  if (mrc != GKS_OK) return mrc;
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
  if (int jrc = join_pipeline(c)) return jrc;
  int mrc = own_mirror(c);
  if (mrc != GKS_OK) return mrc;
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

namespace {
int probe_time_coefs_checked(const double* theta, int n, double dt, double* out, bool single) {
  if (!theta || !out || n < 0) return fail(GKS_EINVAL, "NULL argument or n < 0%s");
  if (!(dt > 0.0) || !std::isfinite(dt)) return fail(GKS_EINVAL, "dt must be finite and > 0%s");
  for (int i = 0; i < n; ++i)
    if (!(theta[i] > 0.0) || !std::isfinite(theta[i])) return fail(GKS_EINVAL, "theta must be finite and > 0%s");
  if (n == 0) return GKS_OK;
  cudaError_t e = gks::probe_time_coefs(theta, n, dt, out, single);
  if (e != cudaSuccess) return cuda_fail(e, "time coefficient probe");
  return GKS_OK;
}
}  // namespace

int gks_probe_time_coefs(const double* theta, int n, double dt, double* out) {
  return probe_time_coefs_checked(theta, n, dt, out, false);
}

int gks_probe_time_coefs_single(const double* theta, int n, double dt, double* out) {
  return probe_time_coefs_checked(theta, n, dt, out, true);
}

int gks_probe_d2f(const double* x, int n, float* out) {
  if (!x || !out || n < 0) return fail(GKS_EINVAL, "NULL argument or n < 0%s");
  if (n == 0) return GKS_OK;
  cudaError_t e = gks::probe_d2f(x, n, out);
  if (e != cudaSuccess) return cuda_fail(e, "conversion probe");
  return GKS_OK;
}

int gks_probe_rcp64(const double* x, int n, double* out) {
  if (!x || !out || n < 0) return fail(GKS_EINVAL, "NULL argument or n < 0%s");
  if (n == 0) return GKS_OK;
  cudaError_t e = gks::probe_rcp64(x, n, out);
  if (e != cudaSuccess) return cuda_fail(e, "reciprocal probe");
  return GKS_OK;
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

int gks_step_host_async(gks_ctx* c, const double* W, const double* Wx, const double* Wy,
                        double* W_out, double* Wx_out, double* Wy_out, double dt) {
  if (!c || !W || !Wx || !W_out || !Wx_out || (c->dim == 2 && (!Wy || !Wy_out)))
    return fail(GKS_EINVAL, "NULL argument%s");
  if (!(dt > 0.0) || !std::isfinite(dt)) return fail(GKS_EINVAL, "dt must be finite and > 0%s");
  const long L = state_len(c);
  const int narr = c->dim + 1;
  const size_t bytes = (size_t)L * sizeof(double);
  cudaError_t e;
  if (!c->slots) {
    e = cudaMalloc(&c->slots, 3 * (size_t)narr * bytes);
    if (e != cudaSuccess) { c->slots = nullptr; return cuda_fail(e, "pipeline slots"); }
    e = cudaStreamCreateWithFlags(&c->s_in, cudaStreamNonBlocking);
    if (e == cudaSuccess) e = cudaStreamCreateWithFlags(&c->s_comp, cudaStreamNonBlocking);
    if (e == cudaSuccess) e = cudaStreamCreateWithFlags(&c->s_out, cudaStreamNonBlocking);
    if (e == cudaSuccess) e = cudaEventCreateWithFlags(&c->ev_ctx, cudaEventDisableTiming);
    for (int k = 0; k < 3 && e == cudaSuccess; ++k) {
      e = cudaEventCreateWithFlags(&c->ev_in[k], cudaEventDisableTiming);
      if (e == cudaSuccess) e = cudaEventCreateWithFlags(&c->ev_done[k], cudaEventDisableTiming);
      if (e == cudaSuccess) e = cudaEventCreateWithFlags(&c->ev_out[k], cudaEventDisableTiming);
      if (e == cudaSuccess) e = cudaEventRecord(c->ev_out[k], c->s_out);
    }
    if (e != cudaSuccess) return cuda_fail(e, "pipeline streams");
  }
  const int k = (int)(c->pipe_calls % 3);
  double* slot = c->slots + (size_t)k * narr * L;
  const double* src[3] = {W, Wx, Wy};
  double* dst[3] = {W_out, Wx_out, Wy_out};
  // copy-in once the slot's previous copy-out (three calls ago) has finished
  e = cudaStreamWaitEvent(c->s_in, c->ev_out[k], 0);
  for (int a = 0; a < narr && e == cudaSuccess; ++a)
    e = cudaMemcpyAsync(slot + a * L, src[a], bytes, cudaMemcpyHostToDevice, c->s_in);
  if (e == cudaSuccess) e = cudaEventRecord(c->ev_in[k], c->s_in);
  if (e != cudaSuccess) return cuda_fail(e, "pipeline copy-in");
  // the step on the pipeline's own stream, after the context's earlier work (which may have
  // replaced the mirror or the step constants) and after the slot's copy-in
  e = cudaEventRecord(c->ev_ctx, c->stream);
  if (e == cudaSuccess) e = cudaStreamWaitEvent(c->s_comp, c->ev_ctx, 0);
  if (e == cudaSuccess) e = cudaStreamWaitEvent(c->s_comp, c->ev_in[k], 0);
  if (e != cudaSuccess) return cuda_fail(e, "pipeline wait");
  cudaStream_t own = c->stream;
  c->stream = c->s_comp;   // the step's launches go to the pipeline stream
  int rc = GKS_OK;
  if (dt != c->last_dt) {
    e = gks::launch_set_times(reinterpret_cast<gks::StepTimes*>(c->d_dt), dt, c->stream);
    if (e != cudaSuccess) rc = cuda_fail(e, "dt update");
    else c->last_dt = dt;
  }
  if (rc == GKS_OK) rc = refresh_mirror(c, slot);
  if (rc == GKS_OK) rc = enqueue_step(c, nullptr, slot);
  c->stream = own;
  if (rc != GKS_OK) return rc;
  e = cudaEventRecord(c->ev_done[k], c->s_comp);
  c->pipe_pending = true;
  c->pipe_last = k;
  // copy-out after the step
  if (e == cudaSuccess) e = cudaStreamWaitEvent(c->s_out, c->ev_done[k], 0);
  for (int a = 0; a < narr && e == cudaSuccess; ++a)
    e = cudaMemcpyAsync(dst[a], slot + a * L, bytes, cudaMemcpyDeviceToHost, c->s_out);
  if (e == cudaSuccess) e = cudaEventRecord(c->ev_out[k], c->s_out);
  if (e != cudaSuccess) return cuda_fail(e, "pipeline copy-out");
  ++c->pipe_calls;
  return GKS_OK;
}

int gks_sync(gks_ctx* c) {
  if (!c) return fail(GKS_EINVAL, "NULL context%s");
  if (c->s_in) {
    cudaError_t e = cudaStreamSynchronize(c->s_in);
    if (e == cudaSuccess) e = cudaStreamSynchronize(c->s_comp);
    if (e == cudaSuccess) e = cudaStreamSynchronize(c->s_out);
    if (e != cudaSuccess) return cuda_fail(e, "pipeline sync");
  }
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
  if (c->s_in) cudaStreamSynchronize(c->s_in);
  if (c->s_comp) cudaStreamSynchronize(c->s_comp);
  if (c->stream) cudaStreamSynchronize(c->stream);
  if (c->s_out) cudaStreamSynchronize(c->s_out);
  for (int k = 0; k < 3; ++k) {
    if (c->ev_in[k]) cudaEventDestroy(c->ev_in[k]);
    if (c->ev_done[k]) cudaEventDestroy(c->ev_done[k]);
    if (c->ev_out[k]) cudaEventDestroy(c->ev_out[k]);
  }
  if (c->ev_ctx) cudaEventDestroy(c->ev_ctx);
  if (c->s_in) cudaStreamDestroy(c->s_in);
  if (c->s_comp) cudaStreamDestroy(c->s_comp);
  if (c->s_out) cudaStreamDestroy(c->s_out);
  if (c->slots) cudaFree(c->slots);
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
