// gks_sweep32.cuh -- FP32-bulk form of the face sweeps and cell updates (device code shared
// by the standalone launches in gks_faces32.cu and the persistent batch kernel in gks_batch.cu).
//
// The reconstruction, WENO-Z and gas-kinetic arithmetic of a face runs in single precision
// on differences from a reference state: the face's left cell (cell f-1 for face f).  The
// state is read from an FP32 mirror that stores every FP64 cell average as a float pair
// hi + lo (hi = float(W), lo = float(W - hi)), so differences of neighbouring cells,
// (hi_k - hi_ref) + (lo_k - lo_ref), keep single-precision accuracy relative to the
// difference.  Slopes are mirrored as floats.
//
// A face evaluates dF = F - F_Euler(W_ref), F_t, W0 - W_ref, W_t and W_tt in single
// precision and writes its flux parts once, in FP64, with the FP64 reference flux added
// (write_face32), and its interface-value parts as single-precision deltas from W_ref; the
// cell update adds W_ref back, so the MSMD accumulation of the cell averages, and
// conservation, stay in FP64.  The slopes at the new time level are difference quotients of
// interface values, formed afresh each step from the FP64 cell difference (rounded) and the
// single-precision interface deltas; they are computed in single precision.  The
// time-integration coefficients of the exponential terms are FP64 (gks_device.cuh).
#pragma once
#include "gks_kernels.cuh"
#include "gks_sweep.cuh"

namespace gks {

// float -> double on the integer pipes: the exponent rebiased (127 -> 1023) and the 23
// significand bits moved to the top of the 52; exact for normal floats, inf and nan, and
// zero; subnormal floats (|f| < 2^-126) become zero of the same sign.  The FP64 pipe also
// executes FP32 -> FP64 conversions and is busy in the stage-2 update and the stage-1
// sweeps; the face epilogues and the updates convert their single-precision parts with this
// instead.
__device__ __forceinline__ double f2d_int(float f) {
  const unsigned b = __float_as_uint(f);
  const unsigned sgn = b & 0x80000000u, e = (b >> 23) & 0xffu, m = b & 0x7fffffu;
  const unsigned ed = e == 0xffu ? 0x7ffu : e + 896u;
  unsigned hi = sgn | (ed << 20) | (m >> 3), lo = m << 29;
  if (e == 0u) { hi = sgn; lo = 0u; }
  return __hiloint2double((int)hi, (int)lo);
}

// f with a subnormal value flushed to zero of the same sign: the float that f2d_int maps to a
// double which converts back to the same float.
__device__ __forceinline__ float ftz_int(float f) {
  const unsigned b = __float_as_uint(f);
  return (b & 0x7f800000u) ? f : __uint_as_float(b & 0x80000000u);
}

// double -> float rounded to nearest (ties to even) on the integer pipes: for results in the
// normal float range the sign, the rebiased exponent (1023 -> 127) and the top 23 fraction
// bits are moved into place and the 29 dropped bits decide the rounding (a carry out of the
// fraction steps the exponent, up to inf); zero, subnormal results, inf and nan take the
// conversion instruction.  Bitwise equal to __double2float_rn (tested through gks_probe_d2f).
__device__ __forceinline__ float d2f_int(double d) {
  const unsigned long long b = (unsigned long long)__double_as_longlong(d);
  const unsigned hi = (unsigned)(b >> 32), lo = (unsigned)b;
  const unsigned e = (hi >> 20) & 0x7ffu;
  if (e < 897u || e > 1150u) return __double2float_rn(d);
  unsigned f = (hi & 0x80000000u) | ((e - 896u) << 23) | ((hi & 0xfffffu) << 3) | (lo >> 29);
  const unsigned rem = lo & 0x1fffffffu;
  f += (rem > 0x10000000u) | ((rem == 0x10000000u) & (f & 1u));
  return __uint_as_float(f);
}

// 1/x for a positive normal x within the float range: a single-precision seed refined by
// two Newton-Raphson steps for f(r) = 1/r - x, r <- r + r (1 - x r), in FP64 (each squares
// the relative error, from ~2^-23 to below FP64 rounding: within a few ulp of 1/x, tested
// through gks_probe_rcp64).  The reference fluxes only; no IEEE rounding guarantee.
__device__ __forceinline__ double rcp64(double x) {
  double r = f2d_int(__frcp_rn((float)x));
  double e = fma(-x, r, 1.0);
  r = fma(r, e, r);
  e = fma(-x, r, 1.0);
  return fma(r, e, r);
}

// Split a binary64 value into floats with w = hi + lo + err, |err| <= 2^-47 |w|, on the
// integer and FP32 pipes: hi is w's significand truncated to 24 bits (a bit copy), lo the
// remaining 29 fraction bits, built exactly in two parts and rounded once to a float by an
// FMA, then scaled by a power of two.  Magnitudes outside [2^-74, 2^128) (zero, tiny, huge)
// take the conversion path.
__device__ __forceinline__ void split_hilo(double w, float& hi, float& lo) {
  const unsigned long long b = (unsigned long long)__double_as_longlong(w);
  const unsigned bh = (unsigned)(b >> 32), bl = (unsigned)b;
  const int e = (int)((bh >> 20) & 0x7ffu);   // biased binary64 exponent
  if (e >= 949 && e <= 1150) {
    const unsigned sign = bh & 0x80000000u;
    hi = __uint_as_float(sign | ((unsigned)(e - 896) << 23) | ((bh & 0xfffffu) << 3) | (bl >> 29));
    const unsigned r = bl & 0x1fffffffu;   // value r * 2^(e - 1075)
    const float rl = __uint_as_float(0x4b000000u | (r & 0x7fffffu)) - 8388608.0f;   // r mod 2^23, exact
    const float rh = __uint_as_float(0x4b000000u | (r >> 23)) - 8388608.0f;         // r / 2^23, exact
    const float rf = fmaf(rh, 8388608.0f, rl);                                     // r rounded to 24 bits
    lo = __uint_as_float(__float_as_uint(rf * __uint_as_float((unsigned)(e - 948) << 23)) | sign);
  } else {
    hi = (float)w;
    lo = (float)(w - (double)hi);
  }
}

// Prefetch of a global line the face epilogue will read (no register is held meanwhile).
// CG (persistent batch kernel): into L2, which is coherent for data written earlier in the
// launch by other SMs; otherwise into L1 (a new launch does not see stale L1 lines).
template <bool CG>
__device__ __forceinline__ void prefetch_line(const void* p) {
  if (CG) asm volatile("prefetch.global.L2 [%0];" ::"l"(p));
  else asm volatile("prefetch.global.L1 [%0];" ::"l"(p));
}

template <int DIM>
__device__ __forceinline__ void swap_uv_f(float* w) {
  if (DIM == 2) { float t = w[1]; w[1] = w[2]; w[2] = t; }
}

// Global loads: CG = true reads through L2 only (__ldcg), for data written earlier in the
// same persistent launch by other blocks (L1 is not coherent across SMs).
template <bool CG>
__device__ __forceinline__ float ldf(const float* p) { return CG ? __ldcg(p) : *p; }
template <bool CG>
__device__ __forceinline__ double ldd(const double* p) { return CG ? __ldcg(p) : *p; }
// one 128-bit load of the four variables of a 2D mirror cell
template <bool CG>
__device__ __forceinline__ float4 ldf4(const float* p) {
  const float4* q = reinterpret_cast<const float4*>(p);
  return CG ? __ldcg(q) : *q;
}
__device__ __forceinline__ void unpack4(const float4 a, float* o) { o[0] = a.x; o[1] = a.y; o[2] = a.z; o[3] = a.w; }

// Layout of the FP32 mirror (blocks q = 0 hi, 1 lo, 2 x slope, 3 y slope): in 2D each block
// is cell-major, the four variables of a cell one float4 (index 4 (q ncell + c) + v), so a
// cell's block is one 128-bit access; in 1D each block is three planes (index
// (3 q + v) ncell + c).  In both, block q starts at q N ncell.
template <int DIM>
__device__ __forceinline__ long mirror_at(int q, int v, long c, long ncell) {
  return DIM == 2 ? 4 * ((long)q * ncell + c) + v : ((long)q * 3 + v) * ncell + c;
}

// Face buffer of the FP32-bulk form: one FP64 block (k = 0 Xi), then five FP32 blocks (q = 0
// dOmega, 1 dLT, 2 A, 3 D, 4 dW), each nfaces long; the FP32 blocks start at FP64 index
// N nfaces (face32_base).  In 2D each block is face-major, a face's four variables contiguous
// (two 128-bit accesses for the FP64 block, one for each FP32 one); in 1D each block is three
// planes.
template <int DIM, bool CG>
__device__ __forceinline__ void ld_face64(const double* o64, int k, long face, long nfaces, double* v) {
  if constexpr (DIM == 2) {
    const double2* p = reinterpret_cast<const double2*>(o64) + 2 * ((long)k * nfaces + face);
    const double2 a = CG ? __ldcg(p) : p[0], b = CG ? __ldcg(p + 1) : p[1];
    v[0] = a.x; v[1] = a.y; v[2] = b.x; v[3] = b.y;
  } else {
#pragma unroll
    for (int i = 0; i < 3; ++i) v[i] = ldd<CG>(o64 + ((long)k * 3 + i) * nfaces + face);
  }
}
template <int DIM>
__device__ __forceinline__ void st_face64(double* o64, int k, long face, long nfaces, const double* v) {
  if constexpr (DIM == 2) {
    double2* p = reinterpret_cast<double2*>(o64) + 2 * ((long)k * nfaces + face);
    p[0] = make_double2(v[0], v[1]);
    p[1] = make_double2(v[2], v[3]);
  } else {
#pragma unroll
    for (int i = 0; i < 3; ++i) o64[((long)k * 3 + i) * nfaces + face] = v[i];
  }
}
template <int DIM, bool CG>
__device__ __forceinline__ void ld_face32(const float* o32, int q, long face, long nfaces, float* v) {
  if constexpr (DIM == 2) {
    unpack4(ldf4<CG>(o32 + 4 * ((long)q * nfaces + face)), v);
  } else {
#pragma unroll
    for (int i = 0; i < 3; ++i) v[i] = ldf<CG>(o32 + ((long)q * 3 + i) * nfaces + face);
  }
}
template <int DIM>
__device__ __forceinline__ void st_face32(float* o32, int q, long face, long nfaces, const float* v) {
  if constexpr (DIM == 2) {
    reinterpret_cast<float4*>(o32)[(long)q * nfaces + face] = make_float4(v[0], v[1], v[2], v[3]);
  } else {
#pragma unroll
    for (int i = 0; i < 3; ++i) o32[((long)q * 3 + i) * nfaces + face] = v[i];
  }
}
template <int DIM>
__device__ __forceinline__ float* face32_base(double* o64, long nfaces) {
  return reinterpret_cast<float*>(o64 + (long)(DIM + 2) * nfaces);
}
template <int DIM>
__device__ __forceinline__ const float* face32_base(const double* o64, long nfaces) {
  return reinterpret_cast<const float*>(o64 + (long)(DIM + 2) * nfaces);
}
template <int DIM>
__device__ __forceinline__ long face64_at(int k, long face, long nfaces) {
  return DIM == 2 ? 4 * ((long)k * nfaces + face) : (long)k * 3 * nfaces + face;
}
template <int DIM>
__device__ __forceinline__ long face32_at(int q, long face, long nfaces) {
  return DIM == 2 ? 4 * ((long)q * nfaces + face) : (long)q * 3 * nfaces + face;
}

// Start the epilogue's global reads of face `face` (stage 1: the FP64 states of its cells
// cl, cr; stage 2: its FP64 flux part Xi and FP32 dLT) while the face is evaluated.
template <int DIM, bool CG>
__device__ __forceinline__ void prefetch_face_epilogue(const FaceArgs32& a, int stage, long face, long nfaces,
                                                       long cl, long cr) {
  const int N = DIM + 2;
  const long ncell = (long)a.nx * a.ny;
  if (stage == 1) {
#pragma unroll
    for (int v = 0; v < N; ++v) { prefetch_line<CG>(a.W + v * ncell + cl); prefetch_line<CG>(a.W + v * ncell + cr); }
  } else {
    const double* o64 = static_cast<const double*>(a.out);
    const float* o32 = face32_base<DIM>(o64, nfaces);
    if constexpr (DIM == 2) {   // a face's Xi and dLT lie in one line each
      prefetch_line<CG>(o64 + face64_at<DIM>(0, face, nfaces));
      prefetch_line<CG>(o32 + face32_at<DIM>(1, face, nfaces));
    } else {
#pragma unroll
      for (int v = 0; v < N; ++v) {
        prefetch_line<CG>(o64 + (long)v * nfaces + face);
        prefetch_line<CG>(o32 + (1L * N + v) * nfaces + face);
      }
    }
  }
}


// Normal Euler flux (global frame) of an FP64 state across a face of direction DIR.
template <int DIM, int DIR>
__device__ __forceinline__ void euler_flux64(const double* W, double gamma, double* F) {
  const int N = DIM + 2;
  const double irho = rcp64(W[0]);
  const double U = W[1] * irho, V = DIM == 2 ? W[2] * irho : 0.0;
  const double p = (gamma - 1.0) * (W[N - 1] - 0.5 * (W[1] * U + (DIM == 2 ? W[2] * V : 0.0)));
  const double un = DIR == 0 ? U : V;
  F[0] = W[1 + DIR];
  F[1] = DIR == 0 ? W[1] * un + p : W[1] * un;
  if (DIM == 2) F[2] = DIR == 1 ? W[2] * un + p : W[2] * un;
  F[N - 1] = (W[N - 1] + p) * un;
}

// Face outputs of the FP32-bulk sweeps.  The face buffer holds one FP64 block, then five FP32
// blocks (layout at ld_face64: per face and block, the variables contiguous in 2D):
//   FP64 Xi  = dt F_ref + (dt dF + dt^2/6 F_t)           (stage 1; stage 2 adds dt^2/3 F_t*)
//   FP32 dOmega = W0 - W_ref + dt/2 W_t + dt^2/8 W_tt     (stage 1)
//   FP32 dLT = W0 - W_ref + dt W_t + dt^2/6 W_tt          (stage 1; stage 2 adds dt^2/3 W_tt*)
//   FP32 A = dt/2 dF + dt^2/8 F_t,  D = dt/2 dFc - A       (stage 1; read by the stage-1 update)
//   FP32 dW  = W_right - W_left of the face's two cells, the FP64 difference rounded (stage 1)
// F_ref = F_Euler(W_left) in FP64 (W_ref = W_left is the face's reference state), dF and F_t the
// single-precision flux delta and derivative, dFc = F_Euler(W_right) - F_Euler(W_left) in the
// single-precision delta form.  Xi is one FP64 value per face, so its differences across a
// cell telescope to FP64 rounding and the FP64 update of the cell averages conserves
// exactly.  The dt/2 flux part only moves the intermediate state W*, so it stays in single
// precision: across cell i its difference is A_{i+1/2} + D_{i-1/2}.  F, Ft, dW0, Wt, Wtt,
// dFc in the global frame; cl, cr: the face's left and right cells.
// STAGE: 1 or 2 fixed at compile time, 0 read from a.stage.
// ml, mr: the left / right cell lies beyond a reflecting wall (its state is the mirror image
// of cell cl / cr, with the momentum normal to the face negated).
template <int DIM, int DIR, bool CG, int STAGE = 0>
__device__ __forceinline__ void write_face32(const FaceArgs32& a, long face, long nfaces, long cl, long cr,
                                             const float* F, const float* Ft, const float* dW0,
                                             const float* Wt, const float* Wtt, const float* dFc,
                                             bool ml = false, bool mr = false) {
  const int N = DIM + 2;
  const long ncell = (long)a.nx * a.ny;
  double* o64 = static_cast<double*>(a.out);
  float* o32 = face32_base<DIM>(o64, nfaces);
  const StepTimes* tc = a.tc;
  const int stage = STAGE ? STAGE : a.stage;
  if (stage == 1) {
    const float hf = ldf<CG>(&tc->hf), h2f = ldf<CG>(&tc->h2f), dtf = ldf<CG>(&tc->dtf), s6f = ldf<CG>(&tc->s6f);
    float dpsi[N], q0[N], q1[N], q2[N], q3[N];
#pragma unroll
    for (int v = 0; v < N; ++v) {
      q0[v] = dW0[v] + hf * Wt[v] + h2f * Wtt[v];
      q1[v] = dW0[v] + dtf * Wt[v] + s6f * Wtt[v];
      q2[v] = hf * F[v] + h2f * Ft[v];
      q3[v] = hf * dFc[v] - q2[v];
      dpsi[v] = dtf * F[v] + s6f * Ft[v];
    }
    st_face32<DIM>(o32, 0, face, nfaces, q0);
    st_face32<DIM>(o32, 1, face, nfaces, q1);
    st_face32<DIM>(o32, 2, face, nfaces, q2);
    st_face32<DIM>(o32, 3, face, nfaces, q3);
    double wl[N], wr[N], Fref[N];
#pragma unroll
    for (int v = 0; v < N; ++v) { wl[v] = ldd<CG>(a.W + v * ncell + cl); wr[v] = ldd<CG>(a.W + v * ncell + cr); }
    if (ml) wl[1 + DIR] = -wl[1 + DIR];
    if (mr) wr[1 + DIR] = -wr[1 + DIR];
    euler_flux64<DIM, DIR>(wl, a.P.gamma, Fref);
    const double dt = ldd<CG>(&tc->dt);
    double xi[N];
    float dw[N];
#pragma unroll
    for (int v = 0; v < N; ++v) {
      // at a wall face every flux but that of the wall-normal momentum is an odd function
      // across the mirror and vanishes; its single-precision delta from the mirrored
      // reference would leave ~1e-8 |rho U| instead, so the FP64 flux is set to zero there
      // (conservation of mass, energy and tangential momentum stays exact)
      const bool odd_at_wall = (ml || mr) && v != 1 + DIR;
      xi[v] = odd_at_wall ? 0.0 : fma(dt, Fref[v], f2d_int(dpsi[v]));
      dw[v] = __double2float_rn(wr[v] - wl[v]);   // the sweep is issue-bound: one conversion
    }
    st_face64<DIM>(o64, 0, face, nfaces, xi);
    st_face32<DIM>(o32, 4, face, nfaces, dw);
  } else {
    const float s3f = ldf<CG>(&tc->s3f);
    double xi[N];
    float lt[N];
    ld_face64<DIM, CG>(o64, 0, face, nfaces, xi);
    ld_face32<DIM, CG>(o32, 1, face, nfaces, lt);
#pragma unroll
    for (int v = 0; v < N; ++v) {
      if (!((ml || mr) && v != 1 + DIR)) xi[v] += f2d_int(s3f * Ft[v]);
      lt[v] += s3f * Wtt[v];
    }
    st_face64<DIM>(o64, 0, face, nfaces, xi);
    st_face32<DIM>(o32, 1, face, nfaces, lt);
  }
}

// ---------------------------------------------------------------------------
// 1D FP32-bulk sweep: one thread per face f = 0..nx.
// ---------------------------------------------------------------------------
// STAGE: 1 or 2 fixed at compile time (stage 2 needs only F_t and W_tt), 0 read from a.stage.
// WALLS: compiled with the reflecting-wall signs (launched for bc 2 only; the periodic and
// transmissive launches carry none of that code).
template <int ORDER, bool WENO, bool VISC, bool CG, int STAGE = 0, bool WALLS = false>
__device__ __forceinline__ void sweep1d_f32_face(const FaceArgs32& a, int f) {
  const int N = 3;
  if (f > a.nx) return;
  const int stage = STAGE ? STAGE : a.stage;
  prefetch_face_epilogue<1, CG>(a, stage, f, a.nx + 1, map_index<WALLS>(f - 1, a.nx, a.bcx), map_index<WALLS>(f, a.nx, a.bcx));
  const double dt = ldd<CG>(a.dtp);
  const long ncell = a.nx;
  const long L = N * ncell;
  float in[N][8], ref[N];
  int cref = map_index<WALLS>(f - 1, a.nx, a.bcx);
  const bool walls = WALLS && a.bcx == 2;
  float rlo[N];
#pragma unroll
  for (int v = 0; v < N; ++v) { ref[v] = ldf<CG>(a.M + v * ncell + cref); rlo[v] = ldf<CG>(a.M + L + v * ncell + cref); }
  if (walls) mirror_ghost<1, 0, float>(ref, rlo, nullptr, beyond_wall(f - 1, a.nx, 2), false);
#pragma unroll
  for (int o = 0; o < 4; ++o) {
    int c = map_index<WALLS>(f - 2 + o, a.nx, a.bcx);
    // cell o = 1 is the reference cell: zero difference, only its slope is loaded
    float hi[N], lo[N], g[N];
#pragma unroll
    for (int v = 0; v < N; ++v) {
      if (o != 1) { hi[v] = ldf<CG>(a.M + v * ncell + c); lo[v] = ldf<CG>(a.M + L + v * ncell + c); }
      else { hi[v] = 0.f; lo[v] = 0.f; }
      g[v] = ldf<CG>(a.Mn + v * ncell + c);
    }
    if (walls) mirror_ghost<1, 0, float>(hi, lo, g, beyond_wall(f - 2 + o, a.nx, 2), false);
#pragma unroll
    for (int v = 0; v < N; ++v) {
      in[v][o] = o == 1 ? 0.f : (hi[v] - ref[v]) + (lo[v] - rlo[v]);
      in[v][4 + o] = a.dnf * g[v];
    }
  }
  float rec[WENO ? 7 : 3][N];
  float dr[N];   // W_right - W_ref
#pragma unroll
  for (int v = 0; v < N; ++v) dr[v] = in[v][2];
  normal_recon<float, 1, ORDER, WENO>(in, a.dnf, a.gammaf, a.epsf, rec, ref);
  PointIn<float, 1> pin;
  float d0[N];
#pragma unroll
  for (int v = 0; v < N; ++v) {
    d0[v] = rec[0][v];
    pin.W0[v] = ref[v] + rec[0][v]; pin.W0x[v] = rec[1][v]; pin.W0xx[v] = rec[2][v];
    pin.Wl[v] = ref[v] + (WENO ? rec[3][v] : rec[0][v]);
    pin.Wlx[v] = WENO ? rec[4][v] : rec[1][v];
    pin.Wr[v] = ref[v] + (WENO ? rec[5][v] : rec[0][v]);
    pin.Wrx[v] = WENO ? rec[6][v] : rec[1][v];
  }
  PointOut<float, 1> po;
  bool ok = gks_point<float, 1, WENO, VISC, true, STAGE != 2>(a.P, pin, dt, po, ref, d0);
  if (!ok) atomicOr(a.status, ST_NONPHYSICAL);
  float dFc[N] = {0.f, 0.f, 0.f};
  if (stage == 1) euler_flux_delta<float, 1>(ref, dr, a.gammaf, dFc);
  write_face32<1, 0, CG, STAGE>(a, f, a.nx + 1, cref, map_index<WALLS>(f, a.nx, a.bcx), po.F, po.Ft, po.W0, po.Wt, po.Wtt, dFc,
                                walls && f == 0, walls && f == a.nx);
}

template <int ORDER, bool WENO, bool VISC, int STAGE, bool WALLS>
__global__ void __launch_bounds__(128) faces_1d_f32_kernel(FaceArgs32 a) {
  sweep1d_f32_face<ORDER, WENO, VISC, false, STAGE, WALLS>(a, blockIdx.x * blockDim.x + threadIdx.x);
}

// ---------------------------------------------------------------------------
// 2D FP32-bulk sweep (same tiling as the FP64 sweep).  Each reconstruction slot keeps its
// reference (hi, lo) in shared memory; the face's Gauss points use the reference of the
// face's own row (tangential slot 2), and the other slots' references enter as
// (hi_t - hi_c) + (lo_t - lo_c).
// Shared memory of the linear Euler tile is slot-major: slot s owns a row of 20 floats, [q][v]
// for the 3 reconstructed quantities of the 4 variables, then the reference hi[4] and lo[4],
// so that one 128-bit shared load brings a quantity of all four variables; 80-byte rows keep
// every 128-bit access of a warp free of bank conflicts (8 consecutive rows fall in distinct
// 16-byte bank groups).  The reference-flux differences follow as one float4 per slot.  The
// WENO-Z / viscous tiles, bound by registers, keep one plane per quantity and variable
// ([q][v][slot], then the reference hi and lo planes and the flux differences) and read them
// one variable at a time.
// ---------------------------------------------------------------------------
constexpr int TA32 = 32, TB32 = 4;   // threads per block: TA32 x TB32

// A tile covers TA32 x (TB32 * FPT) faces: each thread evaluates FPT faces (rows ty, ty + TB32, ...).
template <int DIR, int FPT>
struct Tile32 {
  static constexpr int TB = TB32 * FPT;              // face rows of the tile
  static constexpr int SA = DIR == 0 ? TA32 : TA32 + 4;
  static constexpr int SB = DIR == 0 ? TB + 4 : TB;
  static constexpr int NS = SA * SB;
  // shared memory: per slot NQ reconstructed quantities and the reference (hi, lo), 4 variables
  // each, and the reference-flux difference of the face's two cells (the same size in both
  // layouts)
  static constexpr size_t smem_bytes(bool weno) { return sizeof(float) * (4 * (weno ? 7 : 3) + 12) * NS; }
};

// One tile of TA32 x TB32 faces; tid = linear thread index in a block of TA32 * TB32 threads;
// (bx, by) = tile coordinates (the block indices of the standalone launch); smf = dynamic
// shared memory of Tile32::smem_bytes(WENO) bytes (slot rows, then the slots' reference-flux differences).
// WALLS: as for sweep1d_f32_face.
// TANW: tangential WENO-Z for the non-equilibrium states (option tan_mode 1; WENO-Z tiles).
template <int ORDER, bool WENO, bool VISC, int DIR, bool CG, int FPT = 1, int STAGE = 0, bool WALLS = false,
          bool TANW = false>
__device__ __forceinline__ void sweep2d_f32_tile(const FaceArgs32& a, int bx, int by, int tid, float* smf) {
  const int stage = STAGE ? STAGE : a.stage;
  const int N = 4;
  const int NQ = WENO ? 7 : 3;
  typedef Tile32<DIR, FPT> T;
  const int tx = tid % TA32, ty = tid / TA32;
  constexpr bool AOS = !(WENO || VISC);        // slot-major layout (linear Euler tile)
  constexpr int RS = 4 * NQ + 8;               // floats per slot row (slot-major layout)
  float4* sdfc = reinterpret_cast<float4*>(smf + RS * T::NS);
  float* sref = smf + NQ * N * T::NS;          // plane layout
  float* sreflo = sref + N * T::NS;
  float* sdfcp = sreflo + N * T::NS;
  const double dt = ldd<CG>(a.dtp);
  const long ncell = (long)a.nx * a.ny;
  const int nthreads = TA32 * TB32;
  const int nn = DIR == 0 ? a.nx + 1 : a.ny + 1;

  // reflecting walls on either axis
  const int bcn = DIR == 0 ? a.bcx : a.bcy, bct = DIR == 0 ? a.bcy : a.bcx;
  const int nnc = DIR == 0 ? a.nx : a.ny, ntc = DIR == 0 ? a.ny : a.nx;
  const bool walls = WALLS && ((bcn == 2) | (bct == 2));
  for (int s = tid; s < T::NS; s += nthreads) {
    int sa = s % T::SA, sb = s / T::SA;
    int fn, ctr;   // normal face index, tangential cell index (before mapping)
    if (DIR == 0) { fn = bx * TA32 + sa; ctr = by * T::TB + sb - 2; }
    else { ctr = bx * TA32 + sa - 2; fn = by * T::TB + sb; }
    const int ct = DIR == 0 ? map_index<WALLS>(ctr, a.ny, a.bcy) : map_index<WALLS>(ctr, a.nx, a.bcx);
    float rec[NQ][N];
    float ref[N], rlo[N], dfc[N] = {0.f, 0.f, 0.f, 0.f};
    if (fn < nn) {
      const bool rt = walls && beyond_wall(ctr, ntc, bct);
      long cr;
      if (DIR == 0) cr = (long)ct * a.nx + map_index<WALLS>(fn - 1, a.nx, a.bcx);
      else cr = (long)map_index<WALLS>(fn - 1, a.ny, a.bcy) * a.nx + ct;
      unpack4(ldf4<CG>(a.M + 4 * cr), ref);
      unpack4(ldf4<CG>(a.M + 4 * (ncell + cr)), rlo);
      if (walls) mirror_ghost<2, DIR, float>(ref, rlo, nullptr, beyond_wall(fn - 1, nnc, bcn), rt);
      if (DIR == 1) { swap_uv_f<2>(ref); swap_uv_f<2>(rlo); }
      float in[N][8];
#pragma unroll
      for (int o = 0; o < 4; ++o) {
        long c;
        if (DIR == 0) c = (long)ct * a.nx + map_index<WALLS>(fn - 2 + o, a.nx, a.bcx);
        else c = (long)map_index<WALLS>(fn - 2 + o, a.ny, a.bcy) * a.nx + ct;
        // cell o = 1 is the reference cell itself (same index map and mirror): its
        // difference from the reference is zero and only its slope is loaded
        float hi[N], lo[N], g[N];
        if (o != 1) {
          unpack4(ldf4<CG>(a.M + 4 * c), hi);
          unpack4(ldf4<CG>(a.M + 4 * (ncell + c)), lo);
        } else {
#pragma unroll
          for (int v = 0; v < N; ++v) { hi[v] = 0.f; lo[v] = 0.f; }
        }
        unpack4(ldf4<CG>(a.Mn + 4 * c), g);
        if (walls) mirror_ghost<2, DIR, float>(hi, lo, g, beyond_wall(fn - 2 + o, nnc, bcn), rt);
        if (DIR == 1) { swap_uv_f<2>(hi); swap_uv_f<2>(lo); swap_uv_f<2>(g); }
#pragma unroll
        for (int v = 0; v < N; ++v) {
          in[v][o] = o == 1 ? 0.f : (hi[v] - ref[v]) + (lo[v] - rlo[v]);
          in[v][4 + o] = a.dnf * g[v];
        }
      }
      float dr[N];   // W_right - W_ref
#pragma unroll
      for (int v = 0; v < N; ++v) dr[v] = in[v][2];
      normal_recon<float, 2, ORDER, WENO>(in, a.dnf, a.gammaf, a.epsf, rec, ref);
      // F_Euler(W_right) - F_Euler(W_ref) of the face's two cells, in the face's frame
      // only the tile's own face rows (not the tangential halo) use it
      const bool own = DIR == 0 ? (sb >= 2 && sb < T::TB + 2) : (sa >= 2 && sa < TA32 + 2);
      if (stage == 1 && own) euler_flux_delta<float, 2>(ref, dr, a.gammaf, dfc);
    } else {
#pragma unroll
      for (int q = 0; q < NQ; ++q)
#pragma unroll
        for (int v = 0; v < N; ++v) rec[q][v] = 0.f;
#pragma unroll
      for (int v = 0; v < N; ++v) { ref[v] = 0.f; rlo[v] = 0.f; }
    }
    if constexpr (AOS) {
      float4* row = reinterpret_cast<float4*>(smf + RS * s);
#pragma unroll
      for (int q = 0; q < NQ; ++q) row[q] = make_float4(rec[q][0], rec[q][1], rec[q][2], rec[q][3]);
      row[NQ] = make_float4(ref[0], ref[1], ref[2], ref[3]);
      row[NQ + 1] = make_float4(rlo[0], rlo[1], rlo[2], rlo[3]);
      sdfc[s] = make_float4(dfc[0], dfc[1], dfc[2], dfc[3]);
    } else {
#pragma unroll
      for (int q = 0; q < NQ; ++q)
#pragma unroll
        for (int v = 0; v < N; ++v) smf[(q * N + v) * T::NS + s] = rec[q][v];
#pragma unroll
      for (int v = 0; v < N; ++v) {
        sref[v * T::NS + s] = ref[v]; sreflo[v * T::NS + s] = rlo[v]; sdfcp[v * T::NS + s] = dfc[v];
      }
    }
  }
  __syncthreads();

#pragma unroll 1
  for (int rep = 0; rep < FPT; ++rep) {
  const int ry = ty + rep * TB32;   // face row of this thread within the tile
  int fn, ct;
  if (DIR == 0) { fn = bx * TA32 + tx; ct = by * T::TB + ry; }
  else { ct = bx * TA32 + tx; fn = by * T::TB + ry; }
  const int nt = DIR == 0 ? a.ny : a.nx;
  if (fn >= nn || ct >= nt) continue;
  {
    const long pf = DIR == 0 ? (long)ct * (a.nx + 1) + fn : (long)fn * a.nx + ct;
    const long pn = DIR == 0 ? (long)a.ny * (a.nx + 1) : (long)(a.ny + 1) * a.nx;
    const long pl = DIR == 0 ? (long)ct * a.nx + map_index<WALLS>(fn - 1, a.nx, a.bcx)
                             : (long)map_index<WALLS>(fn - 1, a.ny, a.bcy) * a.nx + ct;
    const long pr = DIR == 0 ? (long)ct * a.nx + map_index<WALLS>(fn, a.nx, a.bcx)
                             : (long)map_index<WALLS>(fn, a.ny, a.bcy) * a.nx + ct;
    prefetch_face_epilogue<2, CG>(a, stage, pf, pn, pl, pr);
  }
  int slot[5];
#pragma unroll
  for (int t = 0; t < 5; ++t)
    slot[t] = DIR == 0 ? (ry + t) * T::SA + tx : ry * T::SA + tx + t;
  // reference of this face and the other slots' reference offsets
  float ref[N], dref[5][N];
  if constexpr (AOS) {
    const float4* own = reinterpret_cast<const float4*>(smf + RS * slot[2]);
    const float4 rh4 = own[NQ], rl4 = own[NQ + 1];
    const float rh[N] = {rh4.x, rh4.y, rh4.z, rh4.w}, rl[N] = {rl4.x, rl4.y, rl4.z, rl4.w};
#pragma unroll
    for (int t = 0; t < 5; ++t) {
      const float4* rw = reinterpret_cast<const float4*>(smf + RS * slot[t]);
      const float4 h4 = rw[NQ], l4 = rw[NQ + 1];
      const float h[N] = {h4.x, h4.y, h4.z, h4.w}, l[N] = {l4.x, l4.y, l4.z, l4.w};
#pragma unroll
      for (int v = 0; v < N; ++v) dref[t][v] = (h[v] - rh[v]) + (l[v] - rl[v]);
    }
#pragma unroll
    for (int v = 0; v < N; ++v) ref[v] = rh[v];
  } else {
#pragma unroll
    for (int v = 0; v < N; ++v) {
      ref[v] = sref[v * T::NS + slot[2]];
      const float rl = sreflo[v * T::NS + slot[2]];
#pragma unroll
      for (int t = 0; t < 5; ++t)
        dref[t][v] = (sref[v * T::NS + slot[t]] - ref[v]) + (sreflo[v * T::NS + slot[t]] - rl);
    }
  }
  const float it = a.itanf;
  float F[N] = {0}, Ft[N] = {0}, dW0[N] = {0}, Wt[N] = {0}, Wtt[N] = {0};
  bool ok = true;
  // unrolled for the linear Euler tile; the WENO-Z / viscous tiles are register-bound
#pragma unroll ((WENO || VISC) ? 1 : 3)
  for (int g = 0; g < 3; ++g) {
    PointIn<float, 2> pin;
    float d0[N];
    if constexpr (AOS) {
      // tangential quartic at Gauss point g: slot t's quantities of all four variables come
      // in one 128-bit shared load each
      float s0[N] = {0}, s1[N] = {0}, s2[N] = {0}, n0[N] = {0}, n1[N] = {0}, nn0[N] = {0};
#pragma unroll
      for (int t = 0; t < 5; ++t) {
        const float w0 = TWf[g][0][t], w1 = TWf[g][1][t], w2 = TWf[g][2][t];
        const float4* rw = reinterpret_cast<const float4*>(smf + RS * slot[t]);
        const float4 a0 = rw[0], a1 = rw[1], a2 = rw[2];
        const float x0[N] = {a0.x, a0.y, a0.z, a0.w}, x1[N] = {a1.x, a1.y, a1.z, a1.w};
        const float x2[N] = {a2.x, a2.y, a2.z, a2.w};
#pragma unroll
        for (int v = 0; v < N; ++v) {
          const float q0 = x0[v] + dref[t][v];
          s0[v] += w0 * q0; s1[v] += w1 * q0; s2[v] += w2 * q0;
          n0[v] += w0 * x1[v]; n1[v] += w1 * x1[v];
          nn0[v] += w0 * x2[v];
        }
      }
#pragma unroll
      for (int v = 0; v < N; ++v) {
        d0[v] = s0[v];
        pin.W0[v] = ref[v] + s0[v]; pin.W0y[v] = s1[v] * it; pin.W0yy[v] = s2[v] * it * it;
        pin.W0x[v] = n0[v]; pin.W0xy[v] = n1[v] * it; pin.W0xx[v] = nn0[v];
        pin.Wl[v] = pin.W0[v]; pin.Wly[v] = pin.W0y[v]; pin.Wlx[v] = n0[v];
        pin.Wr[v] = pin.W0[v]; pin.Wry[v] = pin.W0y[v]; pin.Wrx[v] = n0[v];
      }
    } else {
#pragma unroll
      for (int v = 0; v < N; ++v) {
        float s0 = 0, s1 = 0, s2 = 0, n0 = 0, n1 = 0, nn0 = 0;
        float l0 = 0, l1 = 0, ln0 = 0, r0 = 0, r1 = 0, rn0 = 0;
#pragma unroll
        for (int t = 0; t < 5; ++t) {
          const float w0 = TWf[g][0][t], w1 = TWf[g][1][t], w2 = TWf[g][2][t];
          float q0 = smf[(0 * N + v) * T::NS + slot[t]] + dref[t][v];
          float q1 = smf[(1 * N + v) * T::NS + slot[t]];
          float q2 = smf[(2 * N + v) * T::NS + slot[t]];
          s0 += w0 * q0; s1 += w1 * q0; s2 += w2 * q0;
          n0 += w0 * q1; n1 += w1 * q1;
          nn0 += w0 * q2;
          if (WENO && !TANW) {
            float ql = smf[(3 * N + v) * T::NS + slot[t]] + dref[t][v];
            float qld = smf[(4 * N + v) * T::NS + slot[t]];
            float qr = smf[(5 * N + v) * T::NS + slot[t]] + dref[t][v];
            float qrd = smf[(6 * N + v) * T::NS + slot[t]];
            l0 += w0 * ql; l1 += w1 * ql; ln0 += w0 * qld;
            r0 += w0 * qr; r1 += w1 * qr; rn0 += w0 * qrd;
          }
        }
        d0[v] = s0;
        pin.W0[v] = ref[v] + s0; pin.W0y[v] = s1 * it; pin.W0yy[v] = s2 * it * it;
        pin.W0x[v] = n0; pin.W0xy[v] = n1 * it; pin.W0xx[v] = nn0;
        if (WENO && TANW) {
          // tangential WENO-Z at the Gauss point for the non-equilibrium states
          float ql[5], qld[5], qr[5], qrd[5];
#pragma unroll
          for (int t = 0; t < 5; ++t) {
            ql[t] = smf[(3 * N + v) * T::NS + slot[t]] + dref[t][v];
            qld[t] = smf[(4 * N + v) * T::NS + slot[t]];
            qr[t] = smf[(5 * N + v) * T::NS + slot[t]] + dref[t][v];
            qrd[t] = smf[(6 * N + v) * T::NS + slot[t]];
          }
          const float eps = a.epsf;
          pin.Wl[v] = ref[v] + tan_weno<float, 0>(ql, g, eps); pin.Wly[v] = tan_weno<float, 1>(ql, g, eps) * it;
          pin.Wlx[v] = tan_weno<float, 0>(qld, g, eps);
          pin.Wr[v] = ref[v] + tan_weno<float, 0>(qr, g, eps); pin.Wry[v] = tan_weno<float, 1>(qr, g, eps) * it;
          pin.Wrx[v] = tan_weno<float, 0>(qrd, g, eps);
        } else if (WENO) {
          pin.Wl[v] = ref[v] + l0; pin.Wly[v] = l1 * it; pin.Wlx[v] = ln0;
          pin.Wr[v] = ref[v] + r0; pin.Wry[v] = r1 * it; pin.Wrx[v] = rn0;
        } else {
          pin.Wl[v] = pin.W0[v]; pin.Wly[v] = pin.W0y[v]; pin.Wlx[v] = n0;
          pin.Wr[v] = pin.W0[v]; pin.Wry[v] = pin.W0y[v]; pin.Wrx[v] = n0;
        }
      }
    }
    PointOut<float, 2> po;
    ok &= gks_point<float, 2, WENO, VISC, true, STAGE != 2>(a.P, pin, dt, po, ref, d0);
    const float wg = GWf[g];
#pragma unroll
    for (int v = 0; v < N; ++v) {
      Ft[v] += wg * po.Ft[v]; Wtt[v] += wg * po.Wtt[v];
      if (STAGE != 2) { F[v] += wg * po.F[v]; dW0[v] += wg * po.W0[v]; Wt[v] += wg * po.Wt[v]; }
    }
  }
  if (!ok) atomicOr(a.status, ST_NONPHYSICAL);
  float dFc[N];   // reference-flux difference of the face's two cells (stage 1; phase A)
  if constexpr (AOS) {
    const float4 d4 = sdfc[slot[2]];
    dFc[0] = d4.x; dFc[1] = d4.y; dFc[2] = d4.z; dFc[3] = d4.w;
  } else {
#pragma unroll
    for (int v = 0; v < N; ++v) dFc[v] = sdfcp[v * T::NS + slot[2]];
  }
  if (DIR == 1) {
    swap_uv_f<2>(F); swap_uv_f<2>(Ft); swap_uv_f<2>(dW0); swap_uv_f<2>(Wt); swap_uv_f<2>(Wtt); swap_uv_f<2>(dFc);
  }
  long face, nfaces;
  if (DIR == 0) { face = (long)ct * (a.nx + 1) + fn; nfaces = (long)a.ny * (a.nx + 1); }
  else { face = (long)fn * a.nx + ct; nfaces = (long)(a.ny + 1) * a.nx; }
  // the face's left (reference) and right cells
  const long cl = DIR == 0 ? (long)ct * a.nx + map_index<WALLS>(fn - 1, a.nx, a.bcx)
                           : (long)map_index<WALLS>(fn - 1, a.ny, a.bcy) * a.nx + ct;
  const long cr = DIR == 0 ? (long)ct * a.nx + map_index<WALLS>(fn, a.nx, a.bcx)
                           : (long)map_index<WALLS>(fn, a.ny, a.bcy) * a.nx + ct;
  write_face32<2, DIR, CG, STAGE>(a, face, nfaces, cl, cr, F, Ft, dW0, Wt, Wtt, dFc,
                                  walls && beyond_wall(fn - 1, nnc, bcn), walls && beyond_wall(fn, nnc, bcn));
  }
}

// Linear Euler tiles: five blocks (20 warps) per SM, measured fastest for both stages (the
// first stage spills a few bytes at that bound); the WENO-Z / viscous tiles are left to the
// compiler.
template <int ORDER, bool WENO, bool VISC, int DIR, int FPT, int STAGE, bool WALLS, bool TANW = false>
__global__ void __launch_bounds__(TA32 * TB32, (WENO || VISC) ? 0 : 5)
faces_2d_f32_kernel(FaceArgs32 a) {
  extern __shared__ float smf[];
  sweep2d_f32_tile<ORDER, WENO, VISC, DIR, false, FPT, STAGE, WALLS, TANW>(a, blockIdx.x, blockIdx.y,
                                                                        threadIdx.y * TA32 + threadIdx.x, smf);
}

// ---------------------------------------------------------------------------
// FP32-bulk cell updates (face data as written by write_face32; face i of a row is the left
// face of cell i, its left cell the mapped cell i-1).
//   Stage 1: W* only as the FP32 mirror read by the stage-2 sweep: this cell's hi/lo mirror
//     of W^n plus the single-precision increment -(A_{i+1/2} + D_{i-1/2})/dx - (..)/dy, added
//     exactly (two-sum) and renormalised; the W* slopes (dW + dOmega_{i+1/2} - dOmega_{i-1/2})/dx
//     as floats.
//   Stage 2: W^{n+1} = W^n - (Xi_{i+1/2} - Xi_{i-1/2})/dx - (..)/dy accumulated in FP64 and
//     the slopes W_x^{n+1} = (dW_{i-1/2} + dLT_{i+1/2} - dLT_{i-1/2})/dx in single precision
//     (stored as their exact FP64 images), written in place (each cell reads only its own
//     state), and the mirror of W^{n+1} exactly as write_mirror builds it from the FP64 state
//     (hi/lo of W, the slopes rounded to float), so a run restarted from its FP64 state
//     continues bit for bit.
// ---------------------------------------------------------------------------
// FP32 mirror of one cell's FP64 state: W as hi/lo float pairs, the slopes as floats.
// Store one cell's mirror blocks (hi, lo, x slope, y slope; the y slope unused in 1D).
template <int DIM>
__device__ __forceinline__ void store_mirror(float* M, long c, long ncell, const float* hi,
                                             const float* lo, const float* sx, const float* sy) {
  if constexpr (DIM == 2) {
    float4* M4 = reinterpret_cast<float4*>(M);
    M4[c] = make_float4(hi[0], hi[1], hi[2], hi[3]);
    M4[ncell + c] = make_float4(lo[0], lo[1], lo[2], lo[3]);
    M4[2 * ncell + c] = make_float4(sx[0], sx[1], sx[2], sx[3]);
    M4[3 * ncell + c] = make_float4(sy[0], sy[1], sy[2], sy[3]);
  } else {
#pragma unroll
    for (int v = 0; v < DIM + 2; ++v) {
      M[mirror_at<1>(0, v, c, ncell)] = hi[v];
      M[mirror_at<1>(1, v, c, ncell)] = lo[v];
      M[mirror_at<1>(2, v, c, ncell)] = sx[v];
    }
  }
}

template <int DIM>
__device__ __forceinline__ void write_mirror(float* M, long c, long ncell, const double* w,
                                             const double* wx, const double* wy) {
  const int N = DIM + 2;
  float hi[N], lo[N], sx[N], sy[N];
#pragma unroll
  for (int v = 0; v < N; ++v) {
    split_hilo(w[v], hi[v], lo[v]);
    sx[v] = d2f_int(wx[v]);
    sy[v] = DIM == 2 ? d2f_int(wy[v]) : 0.f;
  }
  store_mirror<DIM>(M, c, ncell, hi, lo, sx, sy);
}

// Cells [c0, c0 + n) of a state of ncell cells.
template <int DIM>
__global__ void __launch_bounds__(256) mirror_kernel(const double* S, float* M, long ncell, long c0, long n) {
  const int N = DIM + 2;
  const long i = (long)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  const long c = c0 + i;
  const long L = N * ncell;
  double w[N], wx[N], wy[N];
#pragma unroll
  for (int v = 0; v < N; ++v) {
    w[v] = S[v * ncell + c];
    wx[v] = S[L + v * ncell + c];
    wy[v] = DIM == 2 ? S[2 * L + v * ncell + c] : 0.0;
  }
  write_mirror<DIM>(M, c, ncell, w, wx, wy);
}

template <int DIM, int STAGE, bool CG>
__device__ __forceinline__ void update_f32_cell(const UpdateArgs32& a, long c) {
  const int N = DIM + 2;
  const long ncell = (long)a.nx * a.ny;
  if (c >= ncell) return;
  const int j = (int)(c / a.nx), i = (int)(c - (long)j * a.nx);
  const long nfx = (long)a.ny * (a.nx + 1), nfy = (long)(a.ny + 1) * a.nx;
  const long fxl = (long)j * (a.nx + 1) + i, fyb = (long)j * a.nx + i, fyt = fyb + a.nx;
  const long L = N * ncell;
  const double* x64 = reinterpret_cast<const double*>(a.fx);
  const double* y64 = reinterpret_cast<const double*>(a.fy);
  float* x32 = a.fx + 2L * N * nfx;   // after the FP64 block (N values per face)
  float* y32 = DIM == 2 ? a.fy + 2L * N * nfy : nullptr;
  const double idx = a.idx, idy = a.idy;
  const float idxf = d2f_int(idx), idyf = d2f_int(idy);
  float* M = a.M;
  if (STAGE == 1) {
    // all loads first
    float h0[N], lo0[N], Ax[N], Dxv[N], Ol[N], Or[N], dWx[N];
    float Ay[N], Dyv[N], Ob[N], Ot[N], dWy[N];
    if constexpr (DIM == 2) {
      unpack4(ldf4<false>(M + 4 * c), h0);
      unpack4(ldf4<false>(M + 4 * (ncell + c)), lo0);
    } else {
#pragma unroll
      for (int v = 0; v < N; ++v) { h0[v] = M[mirror_at<1>(0, v, c, ncell)]; lo0[v] = M[mirror_at<1>(1, v, c, ncell)]; }
    }
    ld_face32<DIM, CG>(x32, 0, fxl, nfx, Ol);
    ld_face32<DIM, CG>(x32, 0, fxl + 1, nfx, Or);
    ld_face32<DIM, CG>(x32, 2, fxl + 1, nfx, Ax);
    ld_face32<DIM, CG>(x32, 3, fxl, nfx, Dxv);
    ld_face32<DIM, CG>(x32, 4, fxl, nfx, dWx);
    if (DIM == 2) {
      ld_face32<DIM, CG>(y32, 0, fyb, nfy, Ob);
      ld_face32<DIM, CG>(y32, 0, fyt, nfy, Ot);
      ld_face32<DIM, CG>(y32, 2, fyt, nfy, Ay);
      ld_face32<DIM, CG>(y32, 3, fyb, nfy, Dyv);
      ld_face32<DIM, CG>(y32, 4, fyb, nfy, dWy);
    }
    float mh[N], ml[N], mx[N], my[N];   // the W* mirror of this cell
#pragma unroll
    for (int v = 0; v < N; ++v) {
      float inc = (Ax[v] + Dxv[v]) * idxf;   // (A_{i+1/2} + D_{i-1/2}) / dx
      const float wxs = (dWx[v] + (Or[v] - Ol[v])) * idxf;
      float wys = 0.f;
      if (DIM == 2) {
        inc += (Ay[v] + Dyv[v]) * idyf;
        wys = (dWy[v] + (Ot[v] - Ob[v])) * idyf;
      }
      // W* = W + d as hi/lo: exact two-sum of the cell's hi with d, renormalised
      const float d = -inc;
      const float s1 = h0[v] + d;
      const float bb = s1 - h0[v];
      const float lo = lo0[v] + ((h0[v] - (s1 - bb)) + (d - bb));
      const float hi = s1 + lo;
      mh[v] = hi;
      ml[v] = lo - (hi - s1);
      mx[v] = wxs;
      my[v] = wys;
    }
    store_mirror<DIM>(M, c, ncell, mh, ml, mx, my);
  } else {
    // all loads first, then the FP64 accumulation and the stores
    double W0[N], Xl[N], Xr[N], Yb[N], Yt[N];
    float dWx[N], lxl[N], lxr[N], dWy[N], lyb[N], lyt[N];
#pragma unroll
    for (int v = 0; v < N; ++v) W0[v] = ldd<CG>(a.W + v * ncell + c);
    ld_face64<DIM, CG>(x64, 0, fxl, nfx, Xl);
    ld_face64<DIM, CG>(x64, 0, fxl + 1, nfx, Xr);
    ld_face32<DIM, CG>(x32, 4, fxl, nfx, dWx);
    ld_face32<DIM, CG>(x32, 1, fxl + 1, nfx, lxr);
    ld_face32<DIM, CG>(x32, 1, fxl, nfx, lxl);
    if (DIM == 2) {
      ld_face64<DIM, CG>(y64, 0, fyb, nfy, Yb);
      ld_face64<DIM, CG>(y64, 0, fyt, nfy, Yt);
      ld_face32<DIM, CG>(y32, 4, fyb, nfy, dWy);
      ld_face32<DIM, CG>(y32, 1, fyt, nfy, lyt);
      ld_face32<DIM, CG>(y32, 1, fyb, nfy, lyb);
    }
    float mh[N], ml[N], mx[N], my[N];   // the W^{n+1} mirror of this cell
#pragma unroll
    for (int v = 0; v < N; ++v) {
      // The slopes (dW_{i-1/2} + dLT_{i+1/2} - dLT_{i-1/2}) / dx in single precision: each
      // is a fresh difference quotient of interface values (nothing accumulates in it), its
      // dLT parts are single-precision results, and the sweeps read it only as a float.  The
      // state keeps it as the exact FP64 image of its float (subnormals flushed to zero), so
      // the float mirror is again a function of the FP64 state.
      double w = W0[v] - (Xr[v] - Xl[v]) * idx;
      const float sx = ftz_int((dWx[v] + (lxr[v] - lxl[v])) * idxf);
      a.W[L + v * ncell + c] = f2d_int(sx);
      mx[v] = sx;
      my[v] = 0.f;
      if (DIM == 2) {
        w -= (Yt[v] - Yb[v]) * idy;
        const float sy = ftz_int((dWy[v] + (lyt[v] - lyb[v])) * idyf);
        a.W[2 * L + v * ncell + c] = f2d_int(sy);
        my[v] = sy;
      }
      a.W[v * ncell + c] = w;
      split_hilo(w, mh[v], ml[v]);
    }
    store_mirror<DIM>(M, c, ncell, mh, ml, mx, my);
  }
}

// Four blocks of 256 threads per SM (64 registers): the stage-2 update issues all of a cell's
// loads before its FP64 arithmetic, and the extra warps overlap one cell's FP64 work with
// other cells' loads (0.244 against 0.281 ms at 2048^2 with three blocks and 80 registers,
// despite 24 B of spills).
template <int DIM, int STAGE>
__global__ void __launch_bounds__(256, 4) update_f32_kernel(UpdateArgs32 a) {
  update_f32_cell<DIM, STAGE, false>(a, (long)blockIdx.x * blockDim.x + threadIdx.x);
}

// Non-inlined wrappers for the persistent batch kernel: each item kind is one call, so the
// batch kernel's size and register allocation stay bounded instead of inlining every
// variant.  The standalone kernels inline the same bodies; the compiler may contract
// multiply-adds differently in the two, so the two agree to single-precision rounding.
template <int ORDER, bool WENO, bool VISC, int STAGE, bool WALLS = false>
__device__ __noinline__ void sweep1d_f32_face_call(const FaceArgs32& a, int f) {
  sweep1d_f32_face<ORDER, WENO, VISC, true, STAGE, WALLS>(a, f);
}
template <int ORDER, bool WENO, bool VISC, int DIR, int FPT, int STAGE, bool WALLS = false>
__device__ __noinline__ void sweep2d_f32_tile_call(const FaceArgs32& a, int bx, int by, int tid, float* smf) {
  sweep2d_f32_tile<ORDER, WENO, VISC, DIR, true, FPT, STAGE, WALLS>(a, bx, by, tid, smf);
}
template <int DIM, int STAGE>
__device__ __noinline__ void update_f32_cell_call(const UpdateArgs32& a, long c) {
  update_f32_cell<DIM, STAGE, true>(a, c);
}

}  // namespace gks
