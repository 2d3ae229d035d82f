// gks_batch.cuh -- device side of the batched FP32-bulk form (see gks_batch.cu): the problem
// table, the work-list item dispatch and the persistent kernel.  Each tile height (faces per
// thread, FPT) is instantiated in a translation unit of its own (gks_batch_k<FPT>.cu) so that
// they compile in parallel.
#pragma once
#include <cuda_runtime.h>

#include "gks_sweep32.cuh"

namespace gks {

enum : unsigned int { ST_TIMEOUT = 4u };

struct BatchProblem {
  FaceArgs32 ax[2], ay[2];   // x / y sweeps, stage 1 and 2
  UpdateArgs32 up;
  int dim, order, recon;
  int tiles_x, tiles_y, tiles_u;   // items per sweep direction / update (per stage)
  int tbx_x, tbx_y;                // tiles along x of the 2D x / y sweep grids
  unsigned need[4];                // items per phase
};

struct BatchArgs {
  const BatchProblem* probs;
  const int4* items;     // (problem, phase, kind, tile); kind 0 x sweep, 1 y sweep, 2 update
  int nitems;
  unsigned* counter;
  unsigned* done;        // [nprob][4]
  unsigned* status;      // [0]: batch-wide flags (ST_TIMEOUT); [1 + p]: flags of problem p
  long long spin_cycles;
};

// Item dispatch.  CLASS 0: 1D (linear / WENO-Z, Euler) and 2D linear Euler problems;
// CLASS 1: every problem kind (2D WENO-Z, Navier-Stokes); CLASS 2: every problem kind, with
// the sweeps compiled with the reflecting-wall signs (a batch holding a walled problem).
template <int CLASS, int FPT>
__device__ __forceinline__ void run_item(const BatchProblem& P, int phase, int kind, int tile, int tid,
                                         float* smf) {
  const int stage = phase < 2 ? 0 : 1;
  constexpr bool WL = CLASS == 2;
  if (phase == 0 || phase == 2) {
    const FaceArgs32& a = kind == 0 ? P.ax[stage] : P.ay[stage];
    const bool visc = a.P.mu > 0.0;
    if (P.dim == 1) {
      const int base = tile * (TA32 * TB32 * FPT);
#pragma unroll 1
      for (int r = 0; r < FPT; ++r) {
        const int f = base + r * (TA32 * TB32) + tid;
        // the MSMD stage (index 0 / 1) picks the stage-1 / stage-2 instantiation
#define GKS_SWEEP1D(O, WN, VS) \
  (stage == 0 ? sweep1d_f32_face_call<O, WN, VS, 1, WL>(a, f) : sweep1d_f32_face_call<O, WN, VS, 2, WL>(a, f))
        if (P.order == 6) {
          if (P.recon == 0) GKS_SWEEP1D(6, false, false);
          else if (CLASS != 0 && visc) GKS_SWEEP1D(6, true, true);
          else GKS_SWEEP1D(6, true, false);
        } else {
          if (P.recon == 0) GKS_SWEEP1D(8, false, false);
          else if (CLASS != 0 && visc) GKS_SWEEP1D(8, true, true);
          else GKS_SWEEP1D(8, true, false);
        }
      }
#undef GKS_SWEEP1D
      return;
    }
    const int tbx = kind == 0 ? P.tbx_x : P.tbx_y;
    const int bx = tile % tbx, by = tile / tbx;
#define GKS_SWEEP2D(O, WN, VS, D)                                              \
  (stage == 0 ? sweep2d_f32_tile_call<O, WN, VS, D, FPT, 1, WL>(a, bx, by, tid, smf) \
              : sweep2d_f32_tile_call<O, WN, VS, D, FPT, 2, WL>(a, bx, by, tid, smf))
    if (CLASS == 0) {
      if (kind == 0) { if (P.order == 6) GKS_SWEEP2D(6, false, false, 0); else GKS_SWEEP2D(8, false, false, 0); }
      else { if (P.order == 6) GKS_SWEEP2D(6, false, false, 1); else GKS_SWEEP2D(8, false, false, 1); }
    } else {
      const bool weno = P.recon == 1;
      if (kind == 0) {
        if (P.order == 6) {
          if (weno) { if (visc) GKS_SWEEP2D(6, true, true, 0); else GKS_SWEEP2D(6, true, false, 0); }
          else { if (visc) GKS_SWEEP2D(6, false, true, 0); else GKS_SWEEP2D(6, false, false, 0); }
        } else {
          if (weno) { if (visc) GKS_SWEEP2D(8, true, true, 0); else GKS_SWEEP2D(8, true, false, 0); }
          else { if (visc) GKS_SWEEP2D(8, false, true, 0); else GKS_SWEEP2D(8, false, false, 0); }
        }
      } else {
        if (P.order == 6) {
          if (weno) { if (visc) GKS_SWEEP2D(6, true, true, 1); else GKS_SWEEP2D(6, true, false, 1); }
          else { if (visc) GKS_SWEEP2D(6, false, true, 1); else GKS_SWEEP2D(6, false, false, 1); }
        } else {
          if (weno) { if (visc) GKS_SWEEP2D(8, true, true, 1); else GKS_SWEEP2D(8, true, false, 1); }
          else { if (visc) GKS_SWEEP2D(8, false, true, 1); else GKS_SWEEP2D(8, false, false, 1); }
        }
      }
    }
#undef GKS_SWEEP2D
    return;
  }
  // cell updates: FPT x 128 cells per item
  const long base = (long)tile * (TA32 * TB32 * FPT);
#pragma unroll 1
  for (int r = 0; r < FPT; ++r) {
    const long c = base + r * (TA32 * TB32) + tid;
    if (P.dim == 1) {
      if (phase == 1) update_f32_cell_call<1, 1>(P.up, c); else update_f32_cell_call<1, 2>(P.up, c);
    } else {
      if (phase == 1) update_f32_cell_call<2, 1>(P.up, c); else update_f32_cell_call<2, 2>(P.up, c);
    }
  }
}

// Class 0 (1D and 2D linear Euler): five blocks per SM (102 registers) measured fastest.
template <int CLASS, int FPT>
__global__ void __launch_bounds__(TA32 * TB32, CLASS == 0 ? 5 : 0) batch_kernel(BatchArgs b) {
  extern __shared__ float smf[];
  __shared__ int s_item, s_abort, s_skip;
  const int tid = threadIdx.x;
  for (;;) {
    if (tid == 0) {
      const int it = (int)atomicAdd(b.counter, 1u);
      int abort = 0, skip = 0;
      if (it < b.nitems) {
        const int4 w = b.items[it];
        if (w.y > 0) {
          // wait for every item of the previous phase of this problem (bounded)
          const volatile unsigned* flag = b.done + 4 * w.x + (w.y - 1);
          const unsigned need = b.probs[w.x].need[w.y - 1];
          const long long t0 = clock64();
          while (*flag < need) {
            if (clock64() - t0 > b.spin_cycles) { atomicOr(b.status, ST_TIMEOUT); abort = 1; break; }
            __nanosleep(100);
          }
          __threadfence();
        }
        // a problem that has met a non-physical state is frozen: its items only signal
        skip = ((volatile unsigned*)b.status)[1 + w.x] != 0u;
      }
      s_item = it;
      s_abort = abort;
      s_skip = skip;
    }
    __syncthreads();
    const int it = s_item;
    if (it >= b.nitems || s_abort) break;
    const int4 w = b.items[it];
    if (!s_skip) run_item<CLASS, FPT>(b.probs[w.x], w.y, w.z, w.w, tid, smf);
    __threadfence();
    __syncthreads();
    if (tid == 0) atomicAdd(b.done + 4 * w.x + w.y, 1u);
  }
}

template <int CLASS, int FPT>
size_t batch_smem() {
  const size_t s0 = Tile32<0, FPT>::smem_bytes(CLASS != 0), s1 = Tile32<1, FPT>::smem_bytes(CLASS != 0);
  return s0 > s1 ? s0 : s1;
}

typedef void (*BatchKernelFn)(BatchArgs);

// Instantiated in gks_batch_k<FPT>.cu (classes 0 and 1) and gks_batch_w<FPT>.cu (class 2):
// the persistent kernel of class `cls` and its dynamic shared memory.
BatchKernelFn batch_kernel_fpt1(int cls);
BatchKernelFn batch_kernel_fpt2(int cls);
BatchKernelFn batch_kernel_fpt4(int cls);
size_t batch_smem_fpt1(int cls);
size_t batch_smem_fpt2(int cls);
size_t batch_smem_fpt4(int cls);
BatchKernelFn batch_kernel_walls_fpt1();
BatchKernelFn batch_kernel_walls_fpt2();
BatchKernelFn batch_kernel_walls_fpt4();

}  // namespace gks
