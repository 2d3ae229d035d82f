// gks_faces.cuh -- FP64 face sweeps of the compact gas-kinetic scheme (one direction, one
// stage): the kernel templates, instantiated in gks_faces.cu (the default reading of the
// equilibrium coefficients) and gks_faces_cm.cu (their full-product variant, CM = true).
//
// Per face: compact reconstruction along the normal (linear, Sec. 3.1; WENO-Z in
// characteristic variables, Sec. 3.3), then (2D) the tangential quartic through five face
// line-averages to three Gauss points, then the gas-kinetic evaluation of Eq.
// (3rd-simplify-flux) at each point, Gauss-averaged over the face.
//
// Stage 1 writes, per face and conservative variable,
//   comp 0: Phi    = dt/2 F + dt^2/8 F_t       (-> W* by Eq. step-hyper-1)
//   comp 1: Psi    = dt F + dt^2/6 F_t         (-> W^{n+1} part of Eq. step-hyper-2)
//   comp 2: Omega  = W0 + dt/2 W_t + dt^2/8 W_tt   (interface value at t*)
//   comp 3: Lambda = W0 + dt W_t + dt^2/6 W_tt     (interface value at t^{n+1}, stage-1 part)
// Stage 2 writes comp 0 = dt^2/3 F_t* and comp 1 = dt^2/3 W_tt*.
//
// Face buffer layouts: x faces [comp][v][ny][nx+1] (face f at x_{f-1/2}); y faces
// [comp][v][ny+1][nx].
#pragma once
#include <atomic>

#include "gks_kernels.cuh"
#include "gks_sweep.cuh"

namespace gks {

// Write the stage outputs of one face; o = output base, stride = faces per plane.
template <int DIM>
__device__ __forceinline__ void write_face(double* out, long face, long nfaces, int stage, double dt,
                                           const double* F, const double* Ft, const double* W0,
                                           const double* Wt, const double* Wtt) {
  const int N = DIM + 2;
  const double plane = (double)0;   // silence unused warnings in some instantiations
  (void)plane;
  if (stage == 1) {
    const double h = 0.5 * dt, h2 = 0.125 * dt * dt, s6 = dt * dt / 6.0;
#pragma unroll
    for (int v = 0; v < N; ++v) {
      out[(0L * N + v) * nfaces + face] = h * F[v] + h2 * Ft[v];
      out[(1L * N + v) * nfaces + face] = dt * F[v] + s6 * Ft[v];
      out[(2L * N + v) * nfaces + face] = W0[v] + h * Wt[v] + h2 * Wtt[v];
      out[(3L * N + v) * nfaces + face] = W0[v] + dt * Wt[v] + s6 * Wtt[v];
    }
  } else {
    const double s3 = dt * dt / 3.0;
#pragma unroll
    for (int v = 0; v < N; ++v) {
      out[(0L * N + v) * nfaces + face] = s3 * Ft[v];
      out[(1L * N + v) * nfaces + face] = s3 * Wtt[v];
    }
  }
}

// ---------------------------------------------------------------------------
// 1D: one thread per face f = 0..nx (face f at x_{f-1/2}).
// ---------------------------------------------------------------------------
// STAGE (1 or 2): the second MSMD stage needs only F_t and W_tt of each face.
// CM: the full-product equilibrium coefficients (coef_mode 1; Euler only).
template <int ORDER, bool WENO, bool VISC, int STAGE, bool CM = false>
__global__ void __launch_bounds__(128) faces_1d_kernel(FaceArgs a) {
  typedef double R;
  const int N = 3;
  int f = blockIdx.x * blockDim.x + threadIdx.x;
  if (f > a.nx) return;
  const double dt = *a.dtp;
  const long ncell = a.nx;
  R in[N][8];
#pragma unroll
  for (int o = 0; o < 4; ++o) {
    int c = map_index(f - 2 + o, a.nx, a.bcx);
    R w[N], g[N];
#pragma unroll
    for (int v = 0; v < N; ++v) { w[v] = a.W[v * ncell + c]; g[v] = a.Wn[v * ncell + c]; }
    if (a.bcx == 2) mirror_ghost<1, 0, R>(w, nullptr, g, beyond_wall(f - 2 + o, a.nx, 2), false);
    if (beyond_iso(f - 2 + o, a.nx, a.bcx)) {
      const int side = f - 2 + o < 0 ? 0 : 1;
      iso_ghost<1>(w, g, 0, true, a.wallT[side], a.wallU[side], a.P.gamma);
    }
#pragma unroll
    for (int v = 0; v < N; ++v) { in[v][o] = w[v]; in[v][4 + o] = a.dn * g[v]; }
  }
  R rec[WENO ? 7 : 3][N];
  normal_recon<R, 1, ORDER, WENO>(in, R(a.dn), R(a.P.gamma), R(a.P.weno_eps), rec, nullptr);
  PointIn<R, 1> pin;
#pragma unroll
  for (int v = 0; v < N; ++v) {
    pin.W0[v] = rec[0][v]; pin.W0x[v] = rec[1][v]; pin.W0xx[v] = rec[2][v];
    pin.Wl[v] = WENO ? rec[3][v] : rec[0][v];
    pin.Wlx[v] = WENO ? rec[4][v] : rec[1][v];
    pin.Wr[v] = WENO ? rec[5][v] : rec[0][v];
    pin.Wrx[v] = WENO ? rec[6][v] : rec[1][v];
  }
  PointOut<R, 1> po;
  bool ok = gks_point<R, 1, WENO, VISC, false, STAGE != 2, CM>(a.P, pin, dt, po);
  if (!ok) atomicOr(a.status, ST_NONPHYSICAL);
  write_face<1>(a.out, f, a.nx + 1, STAGE, dt, po.F, po.Ft, po.W0, po.Wt, po.Wtt);
}

// ---------------------------------------------------------------------------
// 2D face sweep.  DIR 0: x faces, DIR 1: y faces.  The block covers TA x TB faces.
//   DIR 0: threadIdx.x -> face along x (normal), threadIdx.y -> row (tangential);
//          reconstruction slots (TB+4) x TA (two rows of tangential halo each side).
//   DIR 1: threadIdx.x -> column (tangential), threadIdx.y -> face along y (normal);
//          reconstruction slots TB x (TA+4).
// Both keep threadIdx.x on the contiguous x index, so global loads are coalesced.
// ---------------------------------------------------------------------------
constexpr int TA = 32, TB = 4;

template <int DIR>
struct Tile {
  static constexpr int SA = DIR == 0 ? TA : TA + 4;   // slots along threadIdx.x
  static constexpr int SB = DIR == 0 ? TB + 4 : TB;   // slots along threadIdx.y
  static constexpr int NS = SA * SB;
};

// TANW: tangential WENO-Z for the non-equilibrium states (option tan_mode 1, WENO-Z only),
// compiled into instantiations of its own.
template <int ORDER, bool WENO, bool VISC, int DIR, int STAGE, bool TANW = false, bool CM = false>
__global__ void __launch_bounds__(TA * TB) faces_2d_kernel(FaceArgs a) {
  typedef double R;
  const int N = 4;
  const int NQ = WENO ? 7 : 3;
  typedef Tile<DIR> T;
  extern __shared__ double sm[];   // [NQ][N][NS]
  const double dt = *a.dtp;
  const long ncell = (long)a.nx * a.ny;
  const int tid = threadIdx.y * TA + threadIdx.x;
  const int nthreads = TA * TB;
  // faces along the normal: nx+1 (DIR 0) or ny+1 (DIR 1)
  const int nn = DIR == 0 ? a.nx + 1 : a.ny + 1;

  // ---- phase 1: normal reconstruction of every face of the tile plus tangential halo ----
  // reflecting walls on either axis (uniform over the grid: periodic and transmissive
  // grids skip the mirror signs)
  const int bcn = DIR == 0 ? a.bcx : a.bcy, bct = DIR == 0 ? a.bcy : a.bcx;
  const bool walls = (bcn == 2) | (bct == 2);
  const bool iso = (bcn == 3) | (bct == 3);
  for (int s = tid; s < T::NS; s += nthreads) {
    int sa = s % T::SA, sb = s / T::SA;
    int fn, ctr;   // normal face index, tangential cell index (before mapping)
    if (DIR == 0) { fn = blockIdx.x * TA + sa; ctr = blockIdx.y * TB + sb - 2; }
    else { ctr = blockIdx.x * TA + sa - 2; fn = blockIdx.y * TB + sb; }
    const int ct = DIR == 0 ? map_index(ctr, a.ny, a.bcy) : map_index(ctr, a.nx, a.bcx);
    const int nnc = DIR == 0 ? a.nx : a.ny, ntc = DIR == 0 ? a.ny : a.nx;
    R rec[NQ][N];
    if (fn < nn) {
      R in[N][8];
#pragma unroll
      for (int o = 0; o < 4; ++o) {
        long c;
        if (DIR == 0) c = (long)ct * a.nx + map_index(fn - 2 + o, a.nx, a.bcx);
        else c = (long)map_index(fn - 2 + o, a.ny, a.bcy) * a.nx + ct;
        double w[N], g[N];
#pragma unroll
        for (int v = 0; v < N; ++v) { w[v] = a.W[v * ncell + c]; g[v] = a.Wn[v * ncell + c]; }
        if (walls)
          mirror_ghost<2, DIR, double>(w, nullptr, g, beyond_wall(fn - 2 + o, nnc, bcn),
                                       beyond_wall(ctr, ntc, bct));
        if (iso) {
          // isothermal walls: the x wall's map first, then the y wall's (a corner cell)
          const int ix = DIR == 0 ? fn - 2 + o : ctr, iy = DIR == 0 ? ctr : fn - 2 + o;
          if (beyond_iso(ix, a.nx, a.bcx)) {
            const int k = ix < 0 ? 0 : 1;
            iso_ghost<2>(w, g, 0, DIR == 0, a.wallT[k], a.wallU[k], a.P.gamma);
          }
          if (beyond_iso(iy, a.ny, a.bcy)) {
            const int k = iy < 0 ? 2 : 3;
            iso_ghost<2>(w, g, 1, DIR == 1, a.wallT[k], a.wallU[k], a.P.gamma);
          }
        }
        if (DIR == 1) { swap_uv<2>(w); swap_uv<2>(g); }
#pragma unroll
        for (int v = 0; v < N; ++v) { in[v][o] = w[v]; in[v][4 + o] = a.dn * g[v]; }
      }
      normal_recon<R, 2, ORDER, WENO>(in, R(a.dn), R(a.P.gamma), R(a.P.weno_eps), rec, nullptr);
    } else {
#pragma unroll
      for (int q = 0; q < NQ; ++q)
#pragma unroll
        for (int v = 0; v < N; ++v) rec[q][v] = R(0);
    }
#pragma unroll
    for (int q = 0; q < NQ; ++q)
#pragma unroll
      for (int v = 0; v < N; ++v) sm[(q * N + v) * T::NS + s] = rec[q][v];
  }
  __syncthreads();

  // ---- phase 2: tangential quartic to the Gauss points, gas-kinetic evaluation ----
  int fn, ct;
  if (DIR == 0) { fn = blockIdx.x * TA + threadIdx.x; ct = blockIdx.y * TB + threadIdx.y; }
  else { ct = blockIdx.x * TA + threadIdx.x; fn = blockIdx.y * TB + threadIdx.y; }
  const int nt = DIR == 0 ? a.ny : a.nx;
  if (fn >= nn || ct >= nt) return;
  int slot[5];
#pragma unroll
  for (int t = 0; t < 5; ++t)
    slot[t] = DIR == 0 ? (threadIdx.y + t) * T::SA + threadIdx.x : threadIdx.y * T::SA + threadIdx.x + t;
  const R it = R(1) / R(a.dtan);
  const bool tanw = WENO && TANW;
  double F[N] = {0}, Ft[N] = {0}, W0[N] = {0}, Wt[N] = {0}, Wtt[N] = {0};
  bool ok = true;
#pragma unroll 1
  for (int g = 0; g < 3; ++g) {
    PointIn<R, 2> pin;
#pragma unroll
    for (int v = 0; v < N; ++v) {
      R s0 = 0, s1 = 0, s2 = 0, n0 = 0, n1 = 0, nn0 = 0;
      R l0 = 0, l1 = 0, ln0 = 0, r0 = 0, r1 = 0, rn0 = 0;
#pragma unroll
      for (int t = 0; t < 5; ++t) {
        const R w0 = TW[g][0][t], w1 = TW[g][1][t], w2 = TW[g][2][t];
        R q0 = sm[(0 * N + v) * T::NS + slot[t]];
        R q1 = sm[(1 * N + v) * T::NS + slot[t]];
        R q2 = sm[(2 * N + v) * T::NS + slot[t]];
        s0 += w0 * q0; s1 += w1 * q0; s2 += w2 * q0;
        n0 += w0 * q1; n1 += w1 * q1;
        nn0 += w0 * q2;
        if (WENO) {
          R ql = sm[(3 * N + v) * T::NS + slot[t]];
          R qld = sm[(4 * N + v) * T::NS + slot[t]];
          R qr = sm[(5 * N + v) * T::NS + slot[t]];
          R qrd = sm[(6 * N + v) * T::NS + slot[t]];
          l0 += w0 * ql; l1 += w1 * ql; ln0 += w0 * qld;
          r0 += w0 * qr; r1 += w1 * qr; rn0 += w0 * qrd;
        }
      }
      pin.W0[v] = s0; pin.W0y[v] = s1 * it; pin.W0yy[v] = s2 * it * it;
      pin.W0x[v] = n0; pin.W0xy[v] = n1 * it; pin.W0xx[v] = nn0;
      if (WENO) {
        pin.Wl[v] = l0; pin.Wly[v] = l1 * it; pin.Wlx[v] = ln0;
        pin.Wr[v] = r0; pin.Wry[v] = r1 * it; pin.Wrx[v] = rn0;
        if (tanw) {   // tangential WENO-Z for the non-equilibrium states (option tan_mode 1)
          R ql[5], qld[5], qr[5], qrd[5];
#pragma unroll
          for (int t = 0; t < 5; ++t) {
            ql[t] = sm[(3 * N + v) * T::NS + slot[t]]; qld[t] = sm[(4 * N + v) * T::NS + slot[t]];
            qr[t] = sm[(5 * N + v) * T::NS + slot[t]]; qrd[t] = sm[(6 * N + v) * T::NS + slot[t]];
          }
          const R eps = R(a.P.weno_eps);
          pin.Wl[v] = tan_weno<R, 0>(ql, g, eps); pin.Wly[v] = tan_weno<R, 1>(ql, g, eps) * it;
          pin.Wlx[v] = tan_weno<R, 0>(qld, g, eps);
          pin.Wr[v] = tan_weno<R, 0>(qr, g, eps); pin.Wry[v] = tan_weno<R, 1>(qr, g, eps) * it;
          pin.Wrx[v] = tan_weno<R, 0>(qrd, g, eps);
        }
      } else {
        pin.Wl[v] = s0; pin.Wly[v] = s1 * it; pin.Wlx[v] = n0;
        pin.Wr[v] = s0; pin.Wry[v] = s1 * it; pin.Wrx[v] = n0;
      }
    }
    PointOut<R, 2> po;
    ok &= gks_point<R, 2, WENO, VISC, false, STAGE != 2, CM>(a.P, pin, dt, po);
    const double wg = GW[g];
#pragma unroll
    for (int v = 0; v < N; ++v) {
      Ft[v] += wg * po.Ft[v]; Wtt[v] += wg * po.Wtt[v];
      if (STAGE != 2) { F[v] += wg * po.F[v]; W0[v] += wg * po.W0[v]; Wt[v] += wg * po.Wt[v]; }
    }
  }
  if (!ok) atomicOr(a.status, ST_NONPHYSICAL);
  if (DIR == 1) { swap_uv<2>(F); swap_uv<2>(Ft); swap_uv<2>(W0); swap_uv<2>(Wt); swap_uv<2>(Wtt); }
  long face, nfaces;
  if (DIR == 0) { face = (long)ct * (a.nx + 1) + fn; nfaces = (long)a.ny * (a.nx + 1); }
  else { face = (long)fn * a.nx + ct; nfaces = (long)(a.ny + 1) * a.nx; }
  write_face<2>(a.out, face, nfaces, STAGE, dt, F, Ft, W0, Wt, Wtt);
}

// ---------------------------------------------------------------------------
// Launch templates
// ---------------------------------------------------------------------------
template <int ORDER, bool WENO, bool VISC, bool CM = false>
inline cudaError_t launch_1d_t(const FaceArgs& a, cudaStream_t s) {
  int threads = 128;
  int blocks = (a.nx + 1 + threads - 1) / threads;
  if (a.stage == 1) faces_1d_kernel<ORDER, WENO, VISC, 1, CM><<<blocks, threads, 0, s>>>(a);
  else faces_1d_kernel<ORDER, WENO, VISC, 2, CM><<<blocks, threads, 0, s>>>(a);
  return cudaGetLastError();
}

template <int ORDER, bool WENO, bool VISC, int DIR, bool TANW, bool CM = false>
inline cudaError_t launch_2d_tw(const FaceArgs& a, cudaStream_t s) {
  typedef Tile<DIR> T;
  const int NQ = WENO ? 7 : 3;
  size_t shmem = sizeof(double) * NQ * 4 * T::NS;
  static std::atomic<unsigned long long> smem_set{0};
  const void* fns[2] = {(const void*)faces_2d_kernel<ORDER, WENO, VISC, DIR, 1, TANW, CM>,
                        (const void*)faces_2d_kernel<ORDER, WENO, VISC, DIR, 2, TANW, CM>};
  cudaError_t e = smem_limit_per_device(smem_set, fns, 2, (int)shmem);
  if (e != cudaSuccess) return e;
  dim3 block(TA, TB);
  dim3 grid;
  if (DIR == 0) grid = dim3((a.nx + 1 + TA - 1) / TA, (a.ny + TB - 1) / TB);
  else grid = dim3((a.nx + TA - 1) / TA, (a.ny + 1 + TB - 1) / TB);
  if (a.stage == 1) faces_2d_kernel<ORDER, WENO, VISC, DIR, 1, TANW, CM><<<grid, block, shmem, s>>>(a);
  else faces_2d_kernel<ORDER, WENO, VISC, DIR, 2, TANW, CM><<<grid, block, shmem, s>>>(a);
  return cudaGetLastError();
}

template <int ORDER, bool WENO, bool VISC, int DIR>
inline cudaError_t launch_2d_t(const FaceArgs& a, cudaStream_t s) {
  if (WENO && a.P.tan_mode == 1) return launch_2d_tw<ORDER, WENO, VISC, DIR, WENO>(a, s);
  return launch_2d_tw<ORDER, WENO, VISC, DIR, false>(a, s);
}

// All default-reading sweeps of one reconstruction order (instantiated in gks_faces.cu for
// the 6th order and gks_faces_o8.cu for the 8th, which compile in parallel).
template <int ORDER>
cudaError_t launch_faces_1d_order(const FaceArgs& a, int recon, bool visc, cudaStream_t s) {
  if (recon == 0) return visc ? launch_1d_t<ORDER, false, true>(a, s) : launch_1d_t<ORDER, false, false>(a, s);
  return visc ? launch_1d_t<ORDER, true, true>(a, s) : launch_1d_t<ORDER, true, false>(a, s);
}
template <int ORDER, bool WENO, bool VISC>
inline cudaError_t launch_2d_dir(const FaceArgs& a, int dir, cudaStream_t s) {
  return dir == 0 ? launch_2d_t<ORDER, WENO, VISC, 0>(a, s) : launch_2d_t<ORDER, WENO, VISC, 1>(a, s);
}
template <int ORDER>
cudaError_t launch_faces_2d_order(const FaceArgs& a, int dir, int recon, bool visc, cudaStream_t s) {
  if (recon == 0) return visc ? launch_2d_dir<ORDER, false, true>(a, dir, s) : launch_2d_dir<ORDER, false, false>(a, dir, s);
  return visc ? launch_2d_dir<ORDER, true, true>(a, dir, s) : launch_2d_dir<ORDER, true, false>(a, dir, s);
}
// 8th order (gks_faces_o8.cu)
cudaError_t launch_faces_1d_o8(const FaceArgs& a, int recon, bool visc, cudaStream_t s);
cudaError_t launch_faces_2d_o8(const FaceArgs& a, int dir, int recon, bool visc, cudaStream_t s);

// full-product variants (gks_faces_cm.cu)
cudaError_t launch_faces_1d_cm(const FaceArgs& a, int order, int recon, cudaStream_t s);
cudaError_t launch_faces_2d_cm(const FaceArgs& a, int dir, int order, int recon, cudaStream_t s);

}  // namespace gks
