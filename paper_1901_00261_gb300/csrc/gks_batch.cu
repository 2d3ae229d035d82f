// gks_batch.cu -- many independent problems of uneven size advanced together (FP32-bulk form).
//
// One step of every problem is one persistent launch over a work-list of tiles:
//   phase 0: stage-1 face sweeps (x and y tiles of every problem)
//   phase 1: stage-1 cell updates
//   phase 2: stage-2 face sweeps
//   phase 3: stage-2 cell updates
// Items are handed out in this order through an atomic counter.  Before an item of phase k
// of problem p runs, its block waits until every item of phase k-1 of p has completed
// (per-problem completion counters).  Every item it waits on was handed out earlier to a
// running block that does not wait on it, so the waits end; each wait is nevertheless
// bounded by a clock budget, after which the kernel records GKS_ETIMEOUT and its blocks
// return.  The launch is cooperative (all blocks co-resident) and the step (counter resets
// + launch) is replayed from a CUDA graph.  Data produced inside the launch is read through
// L2 (__ldcg).  The tiles run the same device functions as the standalone FP32-bulk kernels
// (through non-inlined wrappers); the compiler fuses multiply-adds differently in the two
// kernels, so a problem advanced in a batch agrees with one advanced alone to single-precision
// rounding, and bitwise with itself under any configuration.
//
// Status: each problem has its own flag word.  A problem whose sweep meets a non-physical
// state (rho <= 0 or p <= 0) is frozen from then on (its items only signal completion), so
// one failing problem neither stops nor perturbs the others; it is reported by index.
//
// The autotuner times the persistent launch for each (tile shape, resident blocks per SM)
// candidate on the batch itself and keeps the fastest; the choice is cached per batch shape.
// Tile shapes: 1, 2 or 4 face rows per thread, i.e. 2D sweep tiles of 32 x 4, 32 x 8 or
// 32 x 16 faces (tangential halo overhead 2, 1.5 or 1.25 reconstructions per face against the
// number of items to balance) and 1D / update items of 128, 256 or 512 faces or cells.
#include <cuda_runtime.h>
#include <math.h>
#include <stdio.h>
#include <string.h>
#include <algorithm>
#include <map>
#include <mutex>
#include <string>
#include <vector>

#include "../../include/gks.h"
#include "gks_batch.cuh"

namespace gks {

// Faces (cells) per thread of the tile shapes the autotuner searches: 2D sweep tiles of
// 32 x 4, 32 x 8 and 32 x 16 faces.
constexpr int FPT_CHOICES[3] = {1, 2, 4};
constexpr int NFPT = 3;
inline int fpt_index(int fpt) { return fpt == 1 ? 0 : (fpt == 2 ? 1 : (fpt == 4 ? 2 : -1)); }

BatchKernelFn batch_kernel_fn(int cls, int fpt) {
  if (cls == 2)
    return fpt == 1 ? batch_kernel_walls_fpt1() : (fpt == 2 ? batch_kernel_walls_fpt2() : batch_kernel_walls_fpt4());
  return fpt == 1 ? batch_kernel_fpt1(cls) : (fpt == 2 ? batch_kernel_fpt2(cls) : batch_kernel_fpt4(cls));
}
size_t batch_smem_of(int cls, int fpt) {
  const int c = cls == 2 ? 1 : cls;   // class 2 tiles are class 1's
  return fpt == 1 ? batch_smem_fpt1(c) : (fpt == 2 ? batch_smem_fpt2(c) : batch_smem_fpt4(c));
}

}  // namespace gks

// ===========================================================================
// Host side
// ===========================================================================
namespace {

thread_local std::string g_berr;
int bfail(int code, const std::string& m) { g_berr = m; return code; }
int bcuda(cudaError_t e, const char* where) {
  g_berr = std::string(where) + ": " + cudaGetErrorString(e);
  return e == cudaErrorMemoryAllocation ? GKS_ENOMEM : GKS_ECUDA;
}

struct TuneKey {
  int cls, nprob;
  long cells;
  bool operator<(const TuneKey& o) const {
    if (cls != o.cls) return cls < o.cls;
    if (nprob != o.nprob) return nprob < o.nprob;
    return cells < o.cells;
  }
};
std::mutex g_tune_mutex;
std::map<TuneKey, std::pair<int, int>> g_tune_cache;   // (fpt, blocks per SM)

}  // namespace

struct gks_batch {
  int n = 0, cls = 0;
  std::vector<gks_problem> prob;
  std::vector<gks::BatchProblem> hp;
  std::vector<long> state_off;   // offsets (doubles) of each problem's state in the arena
  std::vector<long> ncell;
  char* arena = nullptr;
  size_t arena_bytes = 0;
  gks::BatchProblem* dprob = nullptr;
  int4* ditems[gks::NFPT] = {nullptr, nullptr, nullptr};   // work-lists for fpt 1, 2, 4
  int nitems[gks::NFPT] = {0, 0, 0};
  unsigned* dcount = nullptr;   // [0] counter, [1..4n] done
  unsigned* dstatus = nullptr;
  double* ddt = nullptr;
  unsigned long long* dws = nullptr;
  std::vector<double> last_dt;
  std::vector<gks::StepTimes> times;   // host copy of the per-problem step constants
  cudaStream_t stream = nullptr;
  bool own_stream = false;
  int fpt = 1, blocks_per_sm = 0, max_blocks_per_sm[gks::NFPT] = {0, 0, 0}, sms = 0;
  bool cooperative = true;
  long long spin_cycles = 4000000000LL;   // wait budget of a dependency (~2 s at 2 GHz)
  cudaGraph_t graph = nullptr;
  cudaGraphExec_t exec = nullptr;
  std::string tune_report;
};

namespace {

size_t align256(size_t x) { return (x + 255) & ~size_t(255); }

int build_items(gks_batch* B, int fpt, std::vector<int4>& items) {
  items.clear();
  // problems in descending size order within a phase (large problems first balances tails)
  std::vector<int> order(B->n);
  for (int i = 0; i < B->n; ++i) order[i] = i;
  std::stable_sort(order.begin(), order.end(), [&](int a, int b) { return B->ncell[a] > B->ncell[b]; });
  for (int phase = 0; phase < 4; ++phase) {
    for (int p : order) {
      const gks::BatchProblem& P = B->hp[p];
      if (phase == 0 || phase == 2) {
        int tx = P.dim == 1 ? (P.ax[0].nx + 1 + 128 * fpt - 1) / (128 * fpt)
                            : P.tbx_x * ((P.ax[0].ny + 4 * fpt - 1) / (4 * fpt));
        for (int t = 0; t < tx; ++t) items.push_back(make_int4(p, phase, 0, t));
        if (P.dim == 2) {
          int ty = P.tbx_y * ((P.ay[0].ny + 1 + 4 * fpt - 1) / (4 * fpt));
          for (int t = 0; t < ty; ++t) items.push_back(make_int4(p, phase, 1, t));
        }
      } else {
        int tu = (int)((B->ncell[p] + 128 * fpt - 1) / (128 * fpt));
        for (int t = 0; t < tu; ++t) items.push_back(make_int4(p, phase, 2, t));
      }
    }
  }
  return GKS_OK;
}

// per-phase item counts of problem p for a given fpt
void fill_need(gks::BatchProblem& P, long ncell, int fpt) {
  unsigned sw;
  if (P.dim == 1) sw = (P.ax[0].nx + 1 + 128 * fpt - 1) / (128 * fpt);
  else sw = P.tbx_x * ((P.ax[0].ny + 4 * fpt - 1) / (4 * fpt)) + P.tbx_y * ((P.ay[0].ny + 1 + 4 * fpt - 1) / (4 * fpt));
  unsigned up = (unsigned)((ncell + 128 * fpt - 1) / (128 * fpt));
  P.need[0] = sw; P.need[1] = up; P.need[2] = sw; P.need[3] = up;
}

int upload_problems(gks_batch* B, int fpt) {
  for (int p = 0; p < B->n; ++p) fill_need(B->hp[p], B->ncell[p], fpt);
  cudaError_t e = cudaMemcpyAsync(B->dprob, B->hp.data(), sizeof(gks::BatchProblem) * B->n, cudaMemcpyHostToDevice, B->stream);
  if (e == cudaSuccess) e = cudaStreamSynchronize(B->stream);
  if (e != cudaSuccess) return bcuda(e, "batch problem upload");
  return GKS_OK;
}

int enqueue_batch_step(gks_batch* B) {
  const int fi = gks::fpt_index(B->fpt);
  cudaError_t e = cudaMemsetAsync(B->dcount, 0, sizeof(unsigned) * (1 + 4 * B->n), B->stream);
  if (e != cudaSuccess) return bcuda(e, "batch counters");
  gks::BatchArgs a;
  a.probs = B->dprob; a.items = B->ditems[fi]; a.nitems = B->nitems[fi];
  a.counter = B->dcount; a.done = B->dcount + 1; a.status = B->dstatus;
  a.spin_cycles = B->spin_cycles;
  int grid = B->sms * B->blocks_per_sm;
  if (grid > a.nitems) grid = a.nitems > 0 ? a.nitems : 1;
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3(grid);
  cfg.blockDim = dim3(gks::TA32 * gks::TB32);
  cfg.dynamicSmemBytes = gks::batch_smem_of(B->cls, B->fpt);
  cfg.stream = B->stream;
  cudaLaunchAttribute attr[1];
  attr[0].id = cudaLaunchAttributeCooperative;
  attr[0].val.cooperative = B->cooperative ? 1 : 0;
  cfg.attrs = attr;
  cfg.numAttrs = 1;
  e = cudaLaunchKernelEx(&cfg, gks::batch_kernel_fn(B->cls, B->fpt), a);
  if (e != cudaSuccess) return bcuda(e, "batch launch");
  return GKS_OK;
}

void drop_graph(gks_batch* B) {
  if (B->exec) { cudaGraphExecDestroy(B->exec); B->exec = nullptr; }
  if (B->graph) { cudaGraphDestroy(B->graph); B->graph = nullptr; }
}

int set_config(gks_batch* B, int fpt, int bps) {
  const int fi = gks::fpt_index(fpt);
  if (fi < 0) return bfail(GKS_EINVAL, "faces per thread must be 1, 2 or 4");
  if (bps < 1 || bps > B->max_blocks_per_sm[fi]) return bfail(GKS_EINVAL, "blocks per SM out of range");
  if (fpt != B->fpt) {
    int rc = upload_problems(B, fpt);
    if (rc != GKS_OK) return rc;
  }
  B->fpt = fpt;
  B->blocks_per_sm = bps;
  drop_graph(B);
  return GKS_OK;
}

// Reads the status words.  only < 0: every problem counts; else only problem `only`.
// Problems that met a non-physical state are reported by index.
int check_bstatus(gks_batch* B, int only = -1) {
  std::vector<unsigned> st(B->n + 1, 0u);
  cudaError_t e = cudaMemcpyAsync(st.data(), B->dstatus, sizeof(unsigned) * (B->n + 1), cudaMemcpyDeviceToHost, B->stream);
  if (e == cudaSuccess) e = cudaStreamSynchronize(B->stream);
  if (e != cudaSuccess) return bcuda(e, "batch status");
  if (st[0] & gks::ST_TIMEOUT) return bfail(GKS_ETIMEOUT, "a batch dependency wait ran out of its budget");
  std::string bad;
  int nbad = 0;
  for (int p = 0; p < B->n; ++p) {
    if (only >= 0 && p != only) continue;
    if (st[1 + p] & gks::ST_NONPHYSICAL) {
      if (nbad < 8) bad += (nbad ? ", " : "") + std::to_string(p);
      ++nbad;
    }
  }
  if (nbad) return bfail(GKS_ENONPHYSICAL, "non-physical interface state (rho <= 0 or p <= 0) in " + std::to_string(nbad) + " problem(s): " + bad + (nbad > 8 ? ", ..." : ""));
  return GKS_OK;
}

}  // namespace

extern "C" {

const char* gks_batch_last_error(void) { return g_berr.c_str(); }

gks_batch* gks_batch_create(int n, const gks_problem* problems, void* stream) {
  g_berr.clear();
  if (n < 1 || !problems) { bfail(GKS_EINVAL, "need n >= 1 problems"); return nullptr; }
  gks_batch* B = new gks_batch();
  B->n = n;
  B->prob.assign(problems, problems + n);
  B->hp.resize(n);
  B->ncell.resize(n);
  B->state_off.resize(n);
  B->last_dt.assign(n, -1.0);
  // validate and lay out the arena
  std::vector<size_t> off_state(n), off_mir(n), off_fx(n), off_fy(n);
  size_t bytes = 0;
  B->cls = 0;
  for (int p = 0; p < n; ++p) {
    const gks_problem& q = problems[p];
    if (q.nx < 5 || q.ny < 1 || (q.ny > 1 && q.ny < 5) || (long)q.nx * q.ny > (1L << 30)) { bfail(GKS_EINVAL, "problem " + std::to_string(p) + ": grid must have nx >= 5 and ny == 1 or ny >= 5"); delete B; return nullptr; }
    if (q.order != 6 && q.order != 8) { bfail(GKS_EINVAL, "problem " + std::to_string(p) + ": order must be 6 or 8"); delete B; return nullptr; }
    if (q.recon != 0 && q.recon != 1) { bfail(GKS_EINVAL, "problem " + std::to_string(p) + ": recon must be 0 or 1"); delete B; return nullptr; }
    if (!(q.gamma > 1.0) || !(q.mu >= 0.0) || !(q.Pr > 0.0) || !(q.x1 > q.x0) || (q.ny > 1 && !(q.y1 > q.y0))) { bfail(GKS_EINVAL, "problem " + std::to_string(p) + ": invalid physics or domain"); delete B; return nullptr; }
    // periodic, transmissive or reflecting walls (isothermal walls run in the single-problem
    // FP64 form only)
    if (q.bc_x < 0 || q.bc_x > 2 || q.bc_y < 0 || q.bc_y > 2) { bfail(GKS_EINVAL, "problem " + std::to_string(p) + ": bc must be 0, 1 or 2"); delete B; return nullptr; }
    const int dim = q.ny > 1 ? 2 : 1, N = dim + 2;
    if (dim == 2 && (q.recon == 1 || q.mu > 0.0)) B->cls = std::max(B->cls, 1);
    if (dim == 1 && q.mu > 0.0) B->cls = std::max(B->cls, 1);
    if (q.bc_x == 2 || (dim == 2 && q.bc_y == 2)) B->cls = 2;   // the kernel with the wall signs
    const long nc = (long)q.nx * q.ny;
    B->ncell[p] = nc;
    const long L = N * nc;
    off_state[p] = bytes; bytes = align256(bytes + sizeof(double) * (dim + 1) * L);
    off_mir[p] = bytes; bytes = align256(bytes + sizeof(float) * (dim + 2) * L);
    off_fx[p] = bytes; bytes = align256(bytes + sizeof(double) * 4 * N * q.ny * (q.nx + 1));
    off_fy[p] = bytes; if (dim == 2) bytes = align256(bytes + sizeof(double) * 4 * N * (q.ny + 1) * q.nx);
  }
  cudaError_t e;
  if (stream) B->stream = (cudaStream_t)stream;
  else {
    e = cudaStreamCreateWithFlags(&B->stream, cudaStreamNonBlocking);
    if (e != cudaSuccess) { bcuda(e, "stream"); delete B; return nullptr; }
    B->own_stream = true;
  }
  e = cudaMalloc((void**)&B->arena, bytes);
  if (e == cudaSuccess) e = cudaMalloc((void**)&B->dprob, sizeof(gks::BatchProblem) * n);
  if (e == cudaSuccess) e = cudaMalloc((void**)&B->dcount, sizeof(unsigned) * (1 + 4 * n));
  if (e == cudaSuccess) e = cudaMalloc((void**)&B->dstatus, sizeof(unsigned) * (n + 1));
  if (e == cudaSuccess) e = cudaMalloc((void**)&B->ddt, sizeof(double) * gks::STEP_TIMES_DOUBLES * n);
  if (e == cudaSuccess) e = cudaMalloc((void**)&B->dws, sizeof(unsigned long long));
  if (e == cudaSuccess) e = cudaMemsetAsync(B->arena, 0, bytes, B->stream);
  if (e == cudaSuccess) e = cudaMemsetAsync(B->dstatus, 0, sizeof(unsigned) * (n + 1), B->stream);
  if (e != cudaSuccess) { bcuda(e, "batch allocation"); gks_batch_destroy(B); return nullptr; }
  B->arena_bytes = bytes;
  for (int p = 0; p < n; ++p) {
    const gks_problem& q = problems[p];
    const int dim = q.ny > 1 ? 2 : 1, N = dim + 2;
    const long nc = B->ncell[p], L = N * nc;
    double* state = reinterpret_cast<double*>(B->arena + off_state[p]);
    float* mir = reinterpret_cast<float*>(B->arena + off_mir[p]);
    double* fx = reinterpret_cast<double*>(B->arena + off_fx[p]);
    double* fy = dim == 2 ? reinterpret_cast<double*>(B->arena + off_fy[p]) : nullptr;
    B->state_off[p] = (long)(off_state[p] / sizeof(double));
    gks::BatchProblem& P = B->hp[p];
    memset(&P, 0, sizeof(P));
    P.dim = dim; P.order = q.order; P.recon = q.recon;
    const double dx = (q.x1 - q.x0) / q.nx, dy = dim == 2 ? (q.y1 - q.y0) / q.ny : 1.0;
    gks::PhysParams ph{};
    ph.gamma = q.gamma;
    ph.K = dim == 1 ? (3.0 - q.gamma) / (q.gamma - 1.0) : (4.0 - 2.0 * q.gamma) / (q.gamma - 1.0);
    ph.mu = q.mu; ph.Pr = q.Pr; ph.eps_tau = 0.01; ph.C_tau = 1.0; ph.weno_eps = 1e-6;
    gks::set_phys_floats(ph);
    for (int st = 0; st < 2; ++st) {
      for (int d = 0; d < 2; ++d) {
        gks::FaceArgs32& a = d == 0 ? P.ax[st] : P.ay[st];
        a.M = mir; a.W = state;
        a.Mn = mir + (2 + d) * L;
        a.out = d == 0 ? (void*)fx : (void*)fy;
        a.dtp = B->ddt + (size_t)gks::STEP_TIMES_DOUBLES * p;   // this problem's step constants
        a.tc = reinterpret_cast<const gks::StepTimes*>(a.dtp);
        a.status = B->dstatus + 1 + p;
        a.nx = q.nx; a.ny = q.ny; a.bcx = q.bc_x; a.bcy = q.bc_y;
        a.dn = d == 0 ? dx : dy; a.dtan = d == 0 ? dy : dx;
        a.dnf = (float)a.dn; a.itanf = (float)(1.0 / a.dtan);
        a.gammaf = (float)q.gamma; a.epsf = 1e-6f;
        a.stage = st + 1;
        a.P = ph;
      }
    }
    gks::UpdateArgs32& u = P.up;
    u.W = state; u.fx = reinterpret_cast<float*>(fx); u.fy = reinterpret_cast<float*>(fy);
    u.M = mir;
    u.nx = q.nx; u.ny = q.ny; u.bcx = q.bc_x; u.bcy = q.bc_y;
    u.idx = 1.0 / dx; u.idy = 1.0 / dy;
    P.tbx_x = (q.nx + 1 + gks::TA32 - 1) / gks::TA32;
    P.tbx_y = (q.nx + gks::TA32 - 1) / gks::TA32;
  }
  // work-lists for both tile shapes
  for (int fi = 0; fi < gks::NFPT; ++fi) {
    std::vector<int4> items;
    build_items(B, gks::FPT_CHOICES[fi], items);
    B->nitems[fi] = (int)items.size();
    e = cudaMalloc((void**)&B->ditems[fi], sizeof(int4) * std::max<size_t>(items.size(), 1));
    if (e == cudaSuccess) e = cudaMemcpyAsync(B->ditems[fi], items.data(), sizeof(int4) * items.size(), cudaMemcpyHostToDevice, B->stream);
    if (e != cudaSuccess) { bcuda(e, "batch work-list"); gks_batch_destroy(B); return nullptr; }
  }
  // occupancy of the persistent kernel for each tile shape
  int dev = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&B->sms, cudaDevAttrMultiProcessorCount, dev);
  int coop = 0;
  cudaDeviceGetAttribute(&coop, cudaDevAttrCooperativeLaunch, dev);
  B->cooperative = coop != 0;
  for (int fi = 0; fi < gks::NFPT; ++fi) {
    const int f = gks::FPT_CHOICES[fi];
    size_t sm = gks::batch_smem_of(B->cls, f);
    e = cudaFuncSetAttribute(gks::batch_kernel_fn(B->cls, f), cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
    if (e == cudaSuccess) e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&B->max_blocks_per_sm[fi], gks::batch_kernel_fn(B->cls, f), gks::TA32 * gks::TB32, sm);
    if (e != cudaSuccess || B->max_blocks_per_sm[fi] < 1) { bcuda(e == cudaSuccess ? cudaErrorInvalidConfiguration : e, "batch occupancy"); gks_batch_destroy(B); return nullptr; }
  }
  B->fpt = 0;
  // cached tuning for this shape, else the default (1 face per thread, full occupancy)
  long cells = 0;
  for (int p = 0; p < n; ++p) cells += B->ncell[p];
  int fpt = 1, bps = B->max_blocks_per_sm[0];
  {
    std::lock_guard<std::mutex> lock(g_tune_mutex);
    auto it = g_tune_cache.find(TuneKey{B->cls, n, cells});
    if (it != g_tune_cache.end()) { fpt = it->second.first; bps = it->second.second; }
  }
  if (set_config(B, fpt, bps) != GKS_OK) { gks_batch_destroy(B); return nullptr; }
  return B;
}

int gks_batch_set_state(gks_batch* B, int i, const double* W, const double* Wx, const double* Wy) {
  if (!B || i < 0 || i >= B->n || !W || !Wx) return bfail(GKS_EINVAL, "bad argument");
  const gks_problem& q = B->prob[i];
  const int dim = q.ny > 1 ? 2 : 1;
  if (dim == 2 && !Wy) return bfail(GKS_EINVAL, "Wy required in 2D");
  const long L = (dim + 2) * B->ncell[i];
  double* state = reinterpret_cast<double*>(B->arena) + B->state_off[i];
  const double* src[3] = {W, Wx, Wy};
  cudaError_t e = cudaSuccess;
  for (int k = 0; k <= dim && e == cudaSuccess; ++k)
    e = cudaMemcpyAsync(state + k * L, src[k], L * sizeof(double), cudaMemcpyHostToDevice, B->stream);
  if (e != cudaSuccess) return bcuda(e, "batch set_state");
  const gks::BatchProblem& P = B->hp[i];
  e = gks::launch_mirror(state, P.up.M, q.nx, q.ny, dim, B->stream);
  if (e == cudaSuccess) e = cudaMemsetAsync(B->dstatus + 1 + i, 0, sizeof(unsigned), B->stream);   // a new state: no longer frozen
  if (e == cudaSuccess) e = cudaStreamSynchronize(B->stream);
  if (e != cudaSuccess) return bcuda(e, "batch set_state");
  return GKS_OK;
}

int gks_batch_get_state(gks_batch* B, int i, double* W, double* Wx, double* Wy) {
  if (!B || i < 0 || i >= B->n || !W || !Wx) return bfail(GKS_EINVAL, "bad argument");
  const gks_problem& q = B->prob[i];
  const int dim = q.ny > 1 ? 2 : 1;
  if (dim == 2 && !Wy) return bfail(GKS_EINVAL, "Wy required in 2D");
  const long L = (dim + 2) * B->ncell[i];
  const double* state = reinterpret_cast<const double*>(B->arena) + B->state_off[i];
  double* dst[3] = {W, Wx, Wy};
  cudaError_t e = cudaSuccess;
  for (int k = 0; k <= dim && e == cudaSuccess; ++k)
    e = cudaMemcpyAsync(dst[k], state + k * L, L * sizeof(double), cudaMemcpyDeviceToHost, B->stream);
  if (e != cudaSuccess) return bcuda(e, "batch get_state");
  return check_bstatus(B, i);
}

int gks_batch_steps(gks_batch* B, const double* dt, int nsteps) {
  if (!B || !dt) return bfail(GKS_EINVAL, "bad argument");
  if (nsteps < 0) return bfail(GKS_EINVAL, "nsteps must be >= 0");
  bool changed = false;
  for (int p = 0; p < B->n; ++p) {
    if (!(dt[p] > 0.0) || !isfinite(dt[p])) return bfail(GKS_EINVAL, "dt must be finite and > 0");
    if (dt[p] != B->last_dt[p]) changed = true;
  }
  cudaError_t e;
  if (changed) {
    // the step constants of every problem, from the host copy kept in the batch
    B->times.resize(B->n);
    for (int p = 0; p < B->n; ++p) B->times[p] = gks::step_times(dt[p]);
    e = cudaMemcpyAsync(B->ddt, B->times.data(), sizeof(gks::StepTimes) * B->n, cudaMemcpyHostToDevice, B->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(B->stream);   // times may be rewritten by the next call
    if (e != cudaSuccess) return bcuda(e, "batch dt");
    B->last_dt.assign(dt, dt + B->n);
  }
  if (nsteps == 0) return GKS_OK;
  for (int attempt = 0; !B->exec && attempt < 2; ++attempt) {
    e = cudaStreamBeginCapture(B->stream, cudaStreamCaptureModeThreadLocal);
    if (e != cudaSuccess) return bcuda(e, "batch capture");
    int rc = enqueue_batch_step(B);
    cudaGraph_t g = nullptr;
    e = cudaStreamEndCapture(B->stream, &g);
    if (rc == GKS_OK && e == cudaSuccess) {
      e = cudaGraphInstantiate(&B->exec, g, 0);
      if (e == cudaSuccess) { B->graph = g; break; }
    }
    if (g) cudaGraphDestroy(g);
    cudaGetLastError();
    // a cooperative launch that cannot be captured falls back to a plain launch sized to
    // the occupancy (the bounded waits still turn any lost co-residency into an error)
    if (!B->cooperative) return rc != GKS_OK ? rc : bcuda(e, "batch capture");
    B->cooperative = false;
  }
  for (int k = 0; k < nsteps; ++k) {
    e = cudaGraphLaunch(B->exec, B->stream);
    if (e != cudaSuccess) return bcuda(e, "batch graph launch");
  }
  return GKS_OK;
}

int gks_batch_step(gks_batch* B, const double* dt) { return gks_batch_steps(B, dt, 1); }

int gks_batch_sync(gks_batch* B) {
  if (!B) return bfail(GKS_EINVAL, "NULL batch");
  return check_bstatus(B);
}

int gks_batch_max_wavespeed(gks_batch* B, double* out) {
  if (!B || !out) return bfail(GKS_EINVAL, "bad argument");
  for (int p = 0; p < B->n; ++p) {
    const gks_problem& q = B->prob[p];
    const int dim = q.ny > 1 ? 2 : 1;
    const double* state = reinterpret_cast<const double*>(B->arena) + B->state_off[p];
    double dx = (q.x1 - q.x0) / q.nx, dy = dim == 2 ? (q.y1 - q.y0) / q.ny : 1.0;
    cudaError_t e = gks::launch_wavespeed(state, q.nx, q.ny, dim, q.gamma, dx, dy, B->dws, B->stream);
    unsigned long long bits = 0;
    if (e == cudaSuccess) e = cudaMemcpyAsync(&bits, B->dws, sizeof(bits), cudaMemcpyDeviceToHost, B->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(B->stream);
    if (e != cudaSuccess) return bcuda(e, "batch wavespeed");
    memcpy(&out[p], &bits, sizeof(double));
  }
  return GKS_OK;
}

int gks_batch_config(gks_batch* B, int* faces_per_thread, int* blocks_per_sm) {
  if (!B) return bfail(GKS_EINVAL, "NULL batch");
  if (faces_per_thread) *faces_per_thread = B->fpt;
  if (blocks_per_sm) *blocks_per_sm = B->blocks_per_sm;
  return GKS_OK;
}

int gks_batch_set_config(gks_batch* B, int faces_per_thread, int blocks_per_sm) {
  if (!B) return bfail(GKS_EINVAL, "NULL batch");
  return set_config(B, faces_per_thread, blocks_per_sm);
}

int gks_batch_autotune(gks_batch* B, const double* dt, int steps, char* report, int report_len) {
  if (!B || !dt || steps < 1) return bfail(GKS_EINVAL, "bad argument");
  // snapshot the states: tuning steps advance them
  const size_t bytes = B->arena_bytes;
  const size_t sbytes = sizeof(unsigned) * (B->n + 1);
  char* snap = nullptr;
  cudaError_t e = cudaMalloc((void**)&snap, bytes + sbytes);
  if (e != cudaSuccess) return bcuda(e, "autotune snapshot");
  e = cudaMemcpyAsync(snap, B->arena, bytes, cudaMemcpyDeviceToDevice, B->stream);
  if (e == cudaSuccess) e = cudaMemcpyAsync(snap + bytes, B->dstatus, sbytes, cudaMemcpyDeviceToDevice, B->stream);
  if (e != cudaSuccess) { cudaFree(snap); return bcuda(e, "autotune snapshot"); }
  cudaEvent_t t0, t1;
  cudaEventCreate(&t0);
  cudaEventCreate(&t1);
  float best = 1e30f;
  int bf = B->fpt, bb = B->blocks_per_sm;
  std::string rep = "fpt bps ms_per_step\n";
  int rc = GKS_OK;
  for (int fi = 0; fi < gks::NFPT && rc == GKS_OK; ++fi) {
    const int fpt = gks::FPT_CHOICES[fi];
    const int maxb = B->max_blocks_per_sm[fi];
    for (int bps = 1; bps <= maxb && rc == GKS_OK; ++bps) {
      rc = set_config(B, fpt, bps);
      if (rc != GKS_OK) break;
      rc = gks_batch_steps(B, dt, 1);   // warm-up (and graph capture)
      if (rc != GKS_OK) break;
      cudaEventRecord(t0, B->stream);
      rc = gks_batch_steps(B, dt, steps);
      cudaEventRecord(t1, B->stream);
      if (rc != GKS_OK) break;
      e = cudaEventSynchronize(t1);
      if (e != cudaSuccess) { rc = bcuda(e, "autotune timing"); break; }
      float ms = 0.f;
      cudaEventElapsedTime(&ms, t0, t1);
      ms /= steps;
      char line[64];
      snprintf(line, sizeof(line), "%d %d %.4f\n", fpt, bps, ms);
      rep += line;
      if (ms < best) { best = ms; bf = fpt; bb = bps; }
    }
  }
  if (rc == GKS_OK) {
    // a problem that turns non-physical while tuning is frozen, as in a normal step; only a
    // timeout or a CUDA error ends the tuning
    rc = check_bstatus(B);
    if (rc == GKS_ENONPHYSICAL) rc = GKS_OK;
  }
  cudaEventDestroy(t0);
  cudaEventDestroy(t1);
  e = cudaMemcpyAsync(B->arena, snap, bytes, cudaMemcpyDeviceToDevice, B->stream);
  if (e == cudaSuccess) e = cudaMemcpyAsync(B->dstatus, snap + bytes, sbytes, cudaMemcpyDeviceToDevice, B->stream);
  cudaError_t e2 = cudaStreamSynchronize(B->stream);
  cudaFree(snap);
  if (rc != GKS_OK) return rc;
  if (e != cudaSuccess || e2 != cudaSuccess) return bcuda(e != cudaSuccess ? e : e2, "autotune restore");
  rc = set_config(B, bf, bb);
  if (rc != GKS_OK) return rc;
  long cells = 0;
  for (int p = 0; p < B->n; ++p) cells += B->ncell[p];
  {
    std::lock_guard<std::mutex> lock(g_tune_mutex);
    g_tune_cache[TuneKey{B->cls, B->n, cells}] = std::make_pair(bf, bb);
  }
  char line[96];
  snprintf(line, sizeof(line), "chosen: fpt %d, blocks per SM %d (%.4f ms per step)\n", bf, bb, best);
  rep += line;
  B->tune_report = rep;
  if (report && report_len > 0) {
    strncpy(report, rep.c_str(), report_len - 1);
    report[report_len - 1] = 0;
  }
  return GKS_OK;
}

int gks_batch_debug_missing_producer(gks_batch* B, int problem, int phase, double wait_seconds) {
  if (!B || problem < 0 || problem >= B->n || phase < 0 || phase > 2 || !(wait_seconds > 0.0) || wait_seconds > 10.0)
    return bfail(GKS_EINVAL, "bad argument");
  B->hp[problem].need[phase] += 1;   // one item more than the work-list holds: never satisfied
  cudaError_t e = cudaMemcpyAsync(B->dprob + problem, &B->hp[problem], sizeof(gks::BatchProblem), cudaMemcpyHostToDevice, B->stream);
  if (e == cudaSuccess) e = cudaStreamSynchronize(B->stream);
  if (e != cudaSuccess) return bcuda(e, "debug hook");
  B->hp[problem].need[phase] -= 1;   // host copy stays correct; set_config re-uploads it
  B->spin_cycles = (long long)(wait_seconds * 2.07e9);
  drop_graph(B);
  return GKS_OK;
}

int gks_batch_problem_status(gks_batch* B, int* out) {
  if (!B || !out) return bfail(GKS_EINVAL, "bad argument");
  std::vector<unsigned> st(B->n + 1, 0u);
  cudaError_t e = cudaMemcpyAsync(st.data(), B->dstatus, sizeof(unsigned) * (B->n + 1), cudaMemcpyDeviceToHost, B->stream);
  if (e == cudaSuccess) e = cudaStreamSynchronize(B->stream);
  if (e != cudaSuccess) return bcuda(e, "batch status");
  for (int p = 0; p < B->n; ++p) out[p] = (st[1 + p] & gks::ST_NONPHYSICAL) ? GKS_ENONPHYSICAL : GKS_OK;
  return (st[0] & gks::ST_TIMEOUT) ? bfail(GKS_ETIMEOUT, "a batch dependency wait ran out of its budget") : GKS_OK;
}

int gks_batch_reset(gks_batch* B) {
  if (!B) return bfail(GKS_EINVAL, "NULL batch");
  cudaError_t e = cudaMemsetAsync(B->dstatus, 0, sizeof(unsigned) * (B->n + 1), B->stream);
  if (e == cudaSuccess) e = cudaStreamSynchronize(B->stream);
  if (e != cudaSuccess) return bcuda(e, "batch reset");
  B->spin_cycles = 4000000000LL;
  int fpt = B->fpt;
  B->fpt = 0;   // force the problem table upload
  return set_config(B, fpt, B->blocks_per_sm);
}

void gks_batch_destroy(gks_batch* B) {
  if (!B) return;
  if (B->stream) cudaStreamSynchronize(B->stream);
  drop_graph(B);
  if (B->arena) cudaFree(B->arena);
  if (B->dprob) cudaFree(B->dprob);
  for (int fi = 0; fi < gks::NFPT; ++fi) if (B->ditems[fi]) cudaFree(B->ditems[fi]);
  if (B->dcount) cudaFree(B->dcount);
  if (B->dstatus) cudaFree(B->dstatus);
  if (B->ddt) cudaFree(B->ddt);
  if (B->dws) cudaFree(B->dws);
  if (B->own_stream && B->stream) cudaStreamDestroy(B->stream);
  delete B;
}

}  // extern "C"
