// gks_sweep.cuh -- helpers shared by the FP64 and FP32-bulk face sweeps: boundary index
// mapping, the tangential quartic weights and the normal reconstruction of one face.
#pragma once
#include "gks_device.cuh"

namespace gks {

// Cell holding the data of index i of a line of n cells.  bc 0 periodic; bc 1 transmissive
// (the boundary cell); bc 2 reflecting wall and bc 3 isothermal wall: the mirror image across
// the wall (index -1 is cell 0, index n is cell n - 1), which mirror_ghost (bc 2) or
// iso_ghost (bc 3) turns into the ghost.  Indices further out than n, which only the
// overhang of a tile beyond the grid reaches and no face uses, are clamped into the grid.
// WALLS = false: a kernel launched only for bc 0 and 1.
template <bool WALLS = true>
__device__ __forceinline__ int map_index(int i, int n, int bc) {
  if (bc == 0) {
    // indices lie within a few cells of [0, n): one add or subtract; the remainder only for
    // the far halo of grids smaller than a tile
    if (i >= n) { i -= n; if (i >= n) i %= n; }
    else if (i < 0) { i += n; if (i < 0) { i %= n; if (i < 0) i += n; } }
    return i;
  }
  if (WALLS && bc >= 2) { if (i < 0) i = -1 - i; else if (i >= n) i = 2 * n - 1 - i; }
  return i < 0 ? 0 : (i >= n ? n - 1 : i);
}

// True when index i of a line of n cells lies beyond a reflecting wall.
__device__ __forceinline__ bool beyond_wall(int i, int n, int bc) {
  return bc == 2 && (unsigned)i >= (unsigned)n;
}

// True when index i of a line of n cells lies beyond an isothermal wall.
__device__ __forceinline__ bool beyond_iso(int i, int n, int bc) {
  return bc == 3 && (unsigned)i >= (unsigned)n;
}

// Ghost of a cell beyond an isothermal no-slip wall normal to axis `axis` (0 = x, 1 = y):
// the mirror cell's primitive state with the same pressure, the normal velocity negated,
// the tangential one reflected through the wall's (u_t -> 2 u_w - u_t) and the temperature
// p/rho reflected through the wall's (T -> 2 T_w - T), density p/T.  w: conservative values
// (global frame), replaced by the ghost's; g: their derivatives along the stencil, which
// crosses the wall when `normal` (then an even quantity's derivative changes sign) and runs
// along it otherwise; replaced by the derivatives of the ghost field.
template <int DIM>
__device__ __forceinline__ void iso_ghost(double* w, double* g, int axis, bool normal, double Tw,
                                          double uw, double gamma) {
  const int N = DIM + 2;
  const double g1 = gamma - 1.0, irho = 1.0 / w[0];
  const double rho = w[0];
  const double u0 = w[1] * irho, u1 = DIM == 2 ? w[2] * irho : 0.0;
  const double ke = 0.5 * (u0 * u0 + u1 * u1);
  const double p = g1 * (w[N - 1] - rho * ke), T = p * irho;
  const double dr = g[0];
  const double du0 = (g[1] - u0 * dr) * irho, du1 = DIM == 2 ? (g[2] - u1 * dr) * irho : 0.0;
  const double dp = g1 * (g[N - 1] - dr * ke - rho * (u0 * du0 + u1 * du1));
  const double dT = (dp - T * dr) * irho;
  const double sn = normal ? -1.0 : 1.0;   // the sign the map gives an even quantity's slope
  // ghost velocity: the normal component negated, the tangential reflected through uw
  double v0, v1, dv0, dv1;
  if (axis == 0) { v0 = -u0; dv0 = -sn * du0; v1 = 2.0 * uw - u1; dv1 = -sn * du1; }
  else { v1 = -u1; dv1 = -sn * du1; v0 = 2.0 * uw - u0; dv0 = -sn * du0; }
  if (DIM == 1) { v1 = 0.0; dv1 = 0.0; }
  const double Tg = 2.0 * Tw - T, dTg = -sn * dT;
  const double pg = p, dpg = sn * dp;
  const double itg = 1.0 / Tg;
  const double rg = pg * itg, drg = (dpg - rg * dTg) * itg;
  const double keg = 0.5 * (v0 * v0 + v1 * v1), dkeg = v0 * dv0 + v1 * dv1;
  w[0] = rg; g[0] = drg;
  w[1] = rg * v0; g[1] = drg * v0 + rg * dv0;
  if (DIM == 2) { w[2] = rg * v1; g[2] = drg * v1 + rg * dv1; }
  w[N - 1] = pg / g1 + rg * keg;
  g[N - 1] = dpg / g1 + drg * keg + rg * dkeg;
}

// Mirror image of a cell beyond a reflecting wall (conservative variables in the global
// frame).  rn: the wall is crossed by the stencil direction DIR (its normal momentum
// 1 + DIR changes sign, and so do the derivatives along DIR of the other variables);
// rt (2D): the wall is crossed along the tangential axis (the momentum 2 - DIR changes
// sign, in the value and in its derivative along DIR).  w: values (and wlo, the low parts
// of a hi/lo pair, or nullptr); g: derivatives along DIR (or nullptr).
template <int DIM, int DIR, typename R>
__device__ __forceinline__ void mirror_ghost(R* w, R* wlo, R* g, bool rn, bool rt) {
  const int N = DIM + 2, an = 1 + DIR, at = 2 - DIR;
  if (rn) {
    w[an] = -w[an];
    if (wlo) wlo[an] = -wlo[an];
    if (g) {
#pragma unroll
      for (int v = 0; v < N; ++v)
        if (v != an) g[v] = -g[v];
    }
  }
  if (DIM == 2 && rt) {
    w[at] = -w[at];
    if (wlo) wlo[at] = -wlo[at];
    if (g) g[at] = -g[at];
  }
}

// Tangential quartic through the averages over the five unit segments centred at -2..2:
// weights of the value, d/ds and d2/ds2 at the Gauss points s = -sqrt(3/5)/2, 0, +sqrt(3/5)/2.
#define GKS_SQ15 3.87298334620741688518
__device__ __constant__ double TW[3][3][5] = {
    {{-11.0 * GKS_SQ15 / 1200 - 3.0 / 800, 29.0 / 600 + 41.0 * GKS_SQ15 / 600, 1093.0 / 1200,
      29.0 / 600 - 41.0 * GKS_SQ15 / 600, -3.0 / 800 + 11.0 * GKS_SQ15 / 1200},
     {GKS_SQ15 / 100 + 1.0 / 15, -19.0 / 30 - 7.0 * GKS_SQ15 / 50, 13.0 * GKS_SQ15 / 50,
      19.0 / 30 - 7.0 * GKS_SQ15 / 50, -1.0 / 15 + GKS_SQ15 / 100},
     {-1.0 / 20 + GKS_SQ15 / 20, 6.0 / 5 - GKS_SQ15 / 10, -23.0 / 10, GKS_SQ15 / 10 + 6.0 / 5,
      -GKS_SQ15 / 20 - 1.0 / 20}},
    {{3.0 / 640, -29.0 / 480, 1067.0 / 960, -29.0 / 480, 3.0 / 640},
     {5.0 / 48, -17.0 / 24, 0.0, 17.0 / 24, -5.0 / 48},
     {-1.0 / 8, 3.0 / 2, -11.0 / 4, 3.0 / 2, -1.0 / 8}},
    {{-3.0 / 800 + 11.0 * GKS_SQ15 / 1200, 29.0 / 600 - 41.0 * GKS_SQ15 / 600, 1093.0 / 1200,
      29.0 / 600 + 41.0 * GKS_SQ15 / 600, -11.0 * GKS_SQ15 / 1200 - 3.0 / 800},
     {1.0 / 15 - GKS_SQ15 / 100, -19.0 / 30 + 7.0 * GKS_SQ15 / 50, -13.0 * GKS_SQ15 / 50,
      7.0 * GKS_SQ15 / 50 + 19.0 / 30, -1.0 / 15 - GKS_SQ15 / 100},
     {-GKS_SQ15 / 20 - 1.0 / 20, GKS_SQ15 / 10 + 6.0 / 5, -23.0 / 10, 6.0 / 5 - GKS_SQ15 / 10,
      -1.0 / 20 + GKS_SQ15 / 20}}};
// three-point Gauss-Legendre weights on the face
__device__ __constant__ double GW[3] = {5.0 / 18, 8.0 / 18, 5.0 / 18};
// single-precision copies for the FP32-bulk sweeps
__device__ __constant__ float TWf[3][3][5] = {
    {{(float)(-11.0 * GKS_SQ15 / 1200 - 3.0 / 800), (float)(29.0 / 600 + 41.0 * GKS_SQ15 / 600), (float)(1093.0 / 1200),
      (float)(29.0 / 600 - 41.0 * GKS_SQ15 / 600), (float)(-3.0 / 800 + 11.0 * GKS_SQ15 / 1200)},
     {(float)(GKS_SQ15 / 100 + 1.0 / 15), (float)(-19.0 / 30 - 7.0 * GKS_SQ15 / 50), (float)(13.0 * GKS_SQ15 / 50),
      (float)(19.0 / 30 - 7.0 * GKS_SQ15 / 50), (float)(-1.0 / 15 + GKS_SQ15 / 100)},
     {(float)(-1.0 / 20 + GKS_SQ15 / 20), (float)(6.0 / 5 - GKS_SQ15 / 10), (float)(-23.0 / 10), (float)(GKS_SQ15 / 10 + 6.0 / 5),
      (float)(-GKS_SQ15 / 20 - 1.0 / 20)}},
    {{(float)(3.0 / 640), (float)(-29.0 / 480), (float)(1067.0 / 960), (float)(-29.0 / 480), (float)(3.0 / 640)},
     {(float)(5.0 / 48), (float)(-17.0 / 24), 0.0f, (float)(17.0 / 24), (float)(-5.0 / 48)},
     {(float)(-1.0 / 8), (float)(3.0 / 2), (float)(-11.0 / 4), (float)(3.0 / 2), (float)(-1.0 / 8)}},
    {{(float)(-3.0 / 800 + 11.0 * GKS_SQ15 / 1200), (float)(29.0 / 600 - 41.0 * GKS_SQ15 / 600), (float)(1093.0 / 1200),
      (float)(29.0 / 600 + 41.0 * GKS_SQ15 / 600), (float)(-11.0 * GKS_SQ15 / 1200 - 3.0 / 800)},
     {(float)(1.0 / 15 - GKS_SQ15 / 100), (float)(-19.0 / 30 + 7.0 * GKS_SQ15 / 50), (float)(-13.0 * GKS_SQ15 / 50),
      (float)(7.0 * GKS_SQ15 / 50 + 19.0 / 30), (float)(-1.0 / 15 - GKS_SQ15 / 100)},
     {(float)(-GKS_SQ15 / 20 - 1.0 / 20), (float)(GKS_SQ15 / 10 + 6.0 / 5), (float)(-23.0 / 10), (float)(6.0 / 5 - GKS_SQ15 / 10),
      (float)(-1.0 / 20 + GKS_SQ15 / 20)}}};
__device__ __constant__ float GWf[3] = {(float)(5.0 / 18), (float)(8.0 / 18), (float)(5.0 / 18)};

// Tangential WENO-Z at the Gauss points (option tan_mode = 1: the initial non-equilibrium
// states across the face, the WENO reconstruction of Sec. 3.3 carried to the tangential
// direction).  Candidates: the quadratics through the averages of the unit segments
// {-2,-1,0}, {-1,0,1}, {0,1,2} (q[0..4] at offsets -2..2).  TQV[g][k][j] / TQD[g][k][j]: weight
// of q[k + j] in candidate k's value / d/ds at Gauss point g (closed forms).  TQLV, TQLD:
// the linear weights that recombine the candidates into the quartic's value / d/ds at the
// outer points and the derivative at the centre; the centre value's linear weights
// (-9/80, 49/40, -9/80) are split into the positive sets TQP (sum 107/40) and TQM (sum 67/40)
// with theta = 3 (Shi, Hu and Shu, J. Comput. Phys. 175, 2002).
#define GKS_TQ_TABLES(T)                                                                           \
  __device__ __constant__ T TQV##_##T[3][3][3] = {                                                \
      {{T(1.0 / 30 - GKS_SQ15 / 20), T(-1.0 / 15 + GKS_SQ15 / 5), T(31.0 / 30 - 3 * GKS_SQ15 / 20)},   \
       {T(1.0 / 30 + GKS_SQ15 / 20), T(14.0 / 15), T(1.0 / 30 - GKS_SQ15 / 20)},                   \
       {T(31.0 / 30 + 3 * GKS_SQ15 / 20), T(-1.0 / 15 - GKS_SQ15 / 5), T(1.0 / 30 + GKS_SQ15 / 20)}},  \
      {{T(-1.0 / 24), T(1.0 / 12), T(23.0 / 24)},                                                  \
       {T(-1.0 / 24), T(13.0 / 12), T(-1.0 / 24)},                                                 \
       {T(23.0 / 24), T(1.0 / 12), T(-1.0 / 24)}},                                                 \
      {{T(1.0 / 30 + GKS_SQ15 / 20), T(-1.0 / 15 - GKS_SQ15 / 5), T(31.0 / 30 + 3 * GKS_SQ15 / 20)},   \
       {T(1.0 / 30 - GKS_SQ15 / 20), T(14.0 / 15), T(1.0 / 30 + GKS_SQ15 / 20)},                   \
       {T(31.0 / 30 - 3 * GKS_SQ15 / 20), T(-1.0 / 15 + GKS_SQ15 / 5), T(1.0 / 30 - GKS_SQ15 / 20)}}}; \
  __device__ __constant__ T TQD##_##T[3][3][3] = {                                                \
      {{T(0.5 - GKS_SQ15 / 10), T(-2.0 + GKS_SQ15 / 5), T(1.5 - GKS_SQ15 / 10)},                    \
       {T(-0.5 - GKS_SQ15 / 10), T(GKS_SQ15 / 5), T(0.5 - GKS_SQ15 / 10)},                           \
       {T(-1.5 - GKS_SQ15 / 10), T(2.0 + GKS_SQ15 / 5), T(-0.5 - GKS_SQ15 / 10)}},                  \
      {{T(0.5), T(-2.0), T(1.5)}, {T(-0.5), T(0.0), T(0.5)}, {T(-1.5), T(2.0), T(-0.5)}},           \
      {{T(0.5 + GKS_SQ15 / 10), T(-2.0 - GKS_SQ15 / 5), T(1.5 + GKS_SQ15 / 10)},                    \
       {T(-0.5 + GKS_SQ15 / 10), T(-GKS_SQ15 / 5), T(0.5 + GKS_SQ15 / 10)},                          \
       {T(-1.5 + GKS_SQ15 / 10), T(2.0 - GKS_SQ15 / 5), T(-0.5 + GKS_SQ15 / 10)}}};                 \
  __device__ __constant__ T TQLV##_##T[3][3] = {                                                  \
      {T(126.0 / 655 + 71 * GKS_SQ15 / 5240), T(403.0 / 655), T(126.0 / 655 - 71 * GKS_SQ15 / 5240)},   \
      {T(0), T(0), T(0)},                                                                          \
      {T(126.0 / 655 - 71 * GKS_SQ15 / 5240), T(403.0 / 655), T(126.0 / 655 + 71 * GKS_SQ15 / 5240)}};  \
  __device__ __constant__ T TQLD##_##T[3][3] = {                                                  \
      {T(29.0 / 60 + 7 * GKS_SQ15 / 60), T(1.0 / 30), T(29.0 / 60 - 7 * GKS_SQ15 / 60)},             \
      {T(5.0 / 24), T(7.0 / 12), T(5.0 / 24)},                                                     \
      {T(29.0 / 60 - 7 * GKS_SQ15 / 60), T(1.0 / 30), T(29.0 / 60 + 7 * GKS_SQ15 / 60)}};
GKS_TQ_TABLES(double)
GKS_TQ_TABLES(float)
#undef GKS_TQ_TABLES

template <typename R> struct TanWenoTables;
template <> struct TanWenoTables<double> {
  __device__ static const double (&V())[3][3][3] { return TQV_double; }
  __device__ static const double (&D())[3][3][3] { return TQD_double; }
  __device__ static const double (&LV())[3][3] { return TQLV_double; }
  __device__ static const double (&LD())[3][3] { return TQLD_double; }
};
template <> struct TanWenoTables<float> {
  __device__ static const float (&V())[3][3][3] { return TQV_float; }
  __device__ static const float (&D())[3][3][3] { return TQD_float; }
  __device__ static const float (&LV())[3][3] { return TQLV_float; }
  __device__ static const float (&LD())[3][3] { return TQLD_float; }
};

// Smoothness indicators of the three candidates, Eq. (smooth-indicator) on unit segments:
// 13/12 (second difference)^2 + 1/4 (first-derivative combination)^2 (Jiang and Shu).
template <typename R>
__device__ __forceinline__ void tan_weno_beta(const R* q, R* beta) {
  const R c13 = R(13.0 / 12.0), c4 = R(0.25);
  R a = q[0] - R(2) * q[1] + q[2], b = q[0] - R(4) * q[1] + R(3) * q[2];
  beta[0] = c13 * a * a + c4 * b * b;
  a = q[1] - R(2) * q[2] + q[3]; b = q[1] - q[3];
  beta[1] = c13 * a * a + c4 * b * b;
  a = q[2] - R(2) * q[3] + q[4]; b = R(3) * q[2] - R(4) * q[3] + q[4];
  beta[2] = c13 * a * a + c4 * b * b;
}

// WENO-Z combination sum_k delta_k p_k of candidate values p[3] with linear weights d[3],
// Eq. (WENO-Z-w) with the five-point reference value Z = |beta_0 - beta_2|.
template <typename R>
__device__ __forceinline__ R tan_weno_combine(const R* p, const R* beta, R Z, R eps, R d0, R d1, R d2) {
  const R a0 = d0 * (R(1) + Z / (beta[0] + eps));
  const R a1 = d1 * (R(1) + Z / (beta[1] + eps));
  const R a2 = d2 * (R(1) + Z / (beta[2] + eps));
  return (a0 * p[0] + a1 * p[1] + a2 * p[2]) / (a0 + a1 + a2);
}

// Tangential WENO-Z value (DER = 0) or d/ds (DER = 1) at Gauss point g of the centre segment
// from the five segment averages q[0..4].
template <typename R, int DER>
__device__ __forceinline__ R tan_weno(const R* q, int g, R eps) {
  typedef TanWenoTables<R> TT;
  R beta[3], p[3];
  tan_weno_beta(q, beta);
  const R Z = fabs(beta[0] - beta[2]);
#pragma unroll
  for (int k = 0; k < 3; ++k) {
    const R(&w)[3] = DER ? TT::D()[g][k] : TT::V()[g][k];
    p[k] = w[0] * q[k] + w[1] * q[k + 1] + w[2] * q[k + 2];
  }
  if (DER || g != 1) {
    const R(&d)[3] = DER ? TT::LD()[g] : TT::LV()[g];
    return tan_weno_combine(p, beta, Z, eps, d[0], d[1], d[2]);
  }
  // centre value: positive sets (9, 196, 9)/214 and (9, 49, 9)/67, recombined as
  // 107/40 u+ - 67/40 u-
  const R up = tan_weno_combine(p, beta, Z, eps, R(9.0 / 214), R(196.0 / 214), R(9.0 / 214));
  const R um = tan_weno_combine(p, beta, Z, eps, R(9.0 / 67), R(49.0 / 67), R(9.0 / 67));
  return R(107.0 / 40) * up - R(67.0 / 40) * um;
}

// ---------------------------------------------------------------------------
// Normal reconstruction of one face from its 4-cell stencil, in the face's local frame.
// in[v][0..3] = W_{i-1..i+2}, in[v][4..7] = dx W'_{i-1..i+2}.
// rec[0] W0, rec[1] dW0/dn, rec[2] d2W0/dn2, rec[3] Wl, rec[4] dWl/dn, rec[5] Wr, rec[6] dWr/dn
// ---------------------------------------------------------------------------
// base != nullptr: in[v][0..3] are differences from the state base (the eigenvectors of the
// characteristic projection are then taken at base + the mean difference).
template <typename R, int DIM, int ORDER, bool WENO>
__device__ __forceinline__ void normal_recon(const R in[DIM + 2][8], R h, R gamma, R eps,
                                             R rec[WENO ? 7 : 3][DIM + 2], const R* base) {
  const int N = DIM + 2;
  const R ih = R(1) / h;
#pragma unroll
  for (int v = 0; v < N; ++v) {
    R val, dh, ddh2;
    linear_recon<R, ORDER>(in[v][0], in[v][1], in[v][2], in[v][3], in[v][4], in[v][5], in[v][6],
                           in[v][7], val, dh, ddh2);
    rec[0][v] = val;
    rec[1][v] = dh * ih;
    rec[2][v] = ddh2 * ih * ih;
  }
  if (WENO) {
    R Wm[N];
#pragma unroll
    for (int v = 0; v < N; ++v) Wm[v] = R(0.5) * (in[v][1] + in[v][2]) + (base ? base[v] : R(0));
    Eig<R, DIM> e = eig_at<R, DIM>(Wm, gamma);
    R q[8][N];
#pragma unroll
    for (int m = 0; m < 8; ++m) {
      R col[N];
#pragma unroll
      for (int v = 0; v < N; ++v) col[v] = in[v][m];
      eig_left<R, DIM>(e, col, q[m]);
    }
    R lv[N], ld[N], rv[N], rd[N];
#pragma unroll
    for (int k = 0; k < N; ++k) {
      weno_left<R, ORDER>(q[0][k], q[1][k], q[2][k], q[3][k], q[4][k], q[5][k], q[6][k], q[7][k],
                          eps, lv[k], ld[k]);
      // right state: mirror about the interface (cells swap, slopes change sign)
      R d;
      weno_left<R, ORDER>(q[3][k], q[2][k], q[1][k], q[0][k], -q[7][k], -q[6][k], -q[5][k],
                          -q[4][k], eps, rv[k], d);
      rd[k] = -d;
    }
    R t[N];
    eig_right<R, DIM>(e, lv, t);
#pragma unroll
    for (int v = 0; v < N; ++v) rec[3][v] = t[v];
    eig_right<R, DIM>(e, ld, t);
#pragma unroll
    for (int v = 0; v < N; ++v) rec[4][v] = t[v] * ih;
    eig_right<R, DIM>(e, rv, t);
#pragma unroll
    for (int v = 0; v < N; ++v) rec[5][v] = t[v];
    eig_right<R, DIM>(e, rd, t);
#pragma unroll
    for (int v = 0; v < N; ++v) rec[6][v] = t[v] * ih;
  }
}

template <int DIM>
__device__ __forceinline__ void swap_uv(double* w) {
  if (DIM == 2) { double t = w[1]; w[1] = w[2]; w[2] = t; }
}

}  // namespace gks
