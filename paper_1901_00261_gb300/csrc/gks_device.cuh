// gks_device.cuh -- device arithmetic of the compact 6th/8th-order gas-kinetic scheme
// (Zhao, Ji, Shyy, Xu, arXiv:1901.00261).  Everything here runs per interface point in
// the interface's local frame (x = face normal); the kernels in gks_kernels.cu stage
// the data and call it.
//
// R is the bulk arithmetic type (double for the FP64 path, float for the FP32-bulk
// form); the time-integration coefficients of the exponential terms are always FP64.
#pragma once
#include <cuda_runtime.h>
#include <math.h>
#include <stdint.h>

namespace gks {

// a / b in the arithmetic type R: the IEEE division for double; for float the fast
// reciprocal-based division (__fdividef, 2 ulp for 2^-126 < |b| < 2^126), inside the error of
// the single-precision form, whose inputs already carry single-precision rounding.
template <typename R> __device__ __forceinline__ R fdiv(R a, R b);
template <> __device__ __forceinline__ double fdiv<double>(double a, double b) { return a / b; }
template <> __device__ __forceinline__ float fdiv<float>(float a, float b) { return __fdividef(a, b); }
// sqrt(x), x > 0, likewise: IEEE for double, x * rsqrtf(x) (a few ulp) for float.
template <typename R> __device__ __forceinline__ R fsqrt(R x);
template <> __device__ __forceinline__ double fsqrt<double>(double x) { return sqrt(x); }
template <> __device__ __forceinline__ float fsqrt<float>(float x) { return x * rsqrtf(x); }

// ---------------------------------------------------------------------------
// Compact linear reconstruction (Sec. 3.1): interface value, first and second
// derivative at x_{i+1/2} from W_{i-1..i+2} and s_k = dx W'_k (printed coefficients of
// Eqs. recons-6th-val, recons-8th-val, recons-6th-deriva, recons-8th-deriva).
// ---------------------------------------------------------------------------
template <typename R, int ORDER>
__device__ __forceinline__ void linear_recon(R Wm, R W0, R W1, R W2, R sm, R s0, R s1, R s2,
                                             R& val, R& dh, R& ddh2) {
  if (ORDER == 6) {
    val = (Wm + R(299) * (W0 + W1) + W2 - R(3) * (sm - s2) + R(111) * (s0 - s1)) * R(1.0 / 600.0);
    dh = (R(3411) * (W1 - W0) + R(3) * (W2 - Wm) + R(11) * (sm + s2) - R(941) * (s0 + s1)) * R(1.0 / 1560.0);
    ddh2 = ((W0 + W1) - (Wm + W2) + R(3) * (sm - s2) + R(51) * (s1 - s0)) * R(1.0 / 40.0);
  } else {
    val = (R(25) * (Wm + W2) + R(185) * (W0 + W1) + R(6) * (sm - s2) + R(102) * (s0 - s1)) * R(1.0 / 420.0);
    dh = (R(270) * (W1 - W0) + R(14) * (W2 - Wm) - R(3) * (sm + s2) - R(99) * (s0 + s1)) * R(1.0 / 108.0);
    ddh2 = (R(4) * ((W0 + W1) - (Wm + W2)) + (s2 - sm) + R(9) * (s1 - s0)) * R(0.25);
  }
}

// ---------------------------------------------------------------------------
// Compact WENO-Z left state at x_{i+1/2} (Sec. 3.3 and the Appendix).  Candidates are
// the Appendix polynomials w(x) = sum A_p (x/dx)^p / p! (A_p = a_p dx^p) about x_i; the
// w_6 operator before A_4 read as '+'.  beta_1 uses the cubic w~1; the candidate slope
// of stencil S_1 is that of the quadratic w_1 (= w_3).  The (A_4)^2 constant of the
// smoothness indicator is the one its definition gives, 87617/80640.
// Returns the value and dx * derivative.
// ---------------------------------------------------------------------------
template <typename R>
struct Cand { R v, d, b; };

template <typename R>
__device__ __forceinline__ Cand<R> cand_eval(R A0, R A1, R A2, R A3, R A4) {
  Cand<R> c;
  c.v = A0 + R(0.5) * A1 + R(0.125) * A2 + R(1.0 / 48.0) * A3 + R(1.0 / 384.0) * A4;
  c.d = A1 + R(0.5) * A2 + R(0.125) * A3 + R(1.0 / 48.0) * A4;
  c.b = A1 * A1 + R(13.0 / 12.0) * A2 * A2 + R(1043.0 / 960.0) * A3 * A3 +
        R(87617.0 / 80640.0) * A4 * A4 + R(1.0 / 12.0) * A1 * A3 + R(7.0 / 80.0) * A2 * A4;
  return c;
}

template <typename R, int ORDER>
__device__ __forceinline__ void weno_left(R Wm, R W0, R W1, R W2, R sm, R s0, R s1, R s2, R eps,
                                          R& val, R& dh) {
  const R z = R(0);
  Cand<R> c0 = cand_eval<R>((Wm + R(11) * W0 + sm) * R(1.0 / 12.0), R(2) * (W0 - Wm) - sm,
                            R(-2) * (Wm - W0 + sm), z, z);
  Cand<R> c3 = cand_eval<R>((R(26) * W0 - Wm - W1) * R(1.0 / 24.0), R(0.5) * (W1 - Wm),
                            Wm - R(2) * W0 + W1, z, z);
  // w~1: only its smoothness indicator is used
  R t1 = (R(-23) * Wm + R(20) * W0 + R(3) * W1 - R(10) * sm) * R(1.0 / 16.0);
  R t2 = Wm - R(2) * W0 + W1;
  R t3 = R(1.5) * (R(3) * Wm - R(4) * W0 + W1 + R(2) * sm);
  R b1 = t1 * t1 + R(13.0 / 12.0) * t2 * t2 + R(1043.0 / 960.0) * t3 * t3 + R(1.0 / 12.0) * t1 * t3;
  Cand<R> c2 = cand_eval<R>((R(43) * W0 + R(16) * W1 - R(11) * W2 + R(6) * s2) * R(1.0 / 48.0),
                            (R(-31) * W0 + R(60) * W1 - R(29) * W2 + R(14) * s2) * R(1.0 / 16.0),
                            (R(5) * W0 - R(16) * W1 + R(11) * W2 - R(6) * s2) * R(0.5),
                            R(1.5) * (R(4) * W1 - W0 - R(3) * W2 + R(2) * s2), z);
  Cand<R> c4 = cand_eval<R>((R(23) * W0 + R(2) * W1 - W2) * R(1.0 / 24.0),
                            (R(-3) * W0 + R(4) * W1 - W2) * R(0.5), W0 - R(2) * W1 + W2, z, z);
  Cand<R> c5 = cand_eval<R>((R(-175) * Wm + R(1148) * W0 - R(13) * W1 - R(54) * sm - R(108) * s0) * R(1.0 / 960.0),
                            (Wm - W1 + R(10) * s0) * R(0.125),
                            (R(19) * Wm - R(20) * W0 + W1 + R(6) * sm + R(12) * s0) * R(0.25),
                            R(-3) * (Wm - W1 + R(2) * s0),
                            R(-6) * (R(5) * Wm - R(4) * W0 - W1 + R(2) * sm + R(4) * s0));
  Cand<R> c6 = cand_eval<R>((R(707) * W0 - R(292) * W1 + R(545) * W2 - R(612) * s1 - R(186) * s2) * R(1.0 / 960.0),
                            (R(-21) * W0 + R(8) * W1 + R(13) * W2 - R(22) * s1 - R(4) * s2) * R(0.125),
                            (R(25) * W0 + R(28) * W1 - R(53) * W2 + R(60) * s1 + R(18) * s2) * R(0.25),
                            R(-3) * (R(3) * W0 + R(8) * W1 - R(11) * W2 + R(10) * s1 + R(4) * s2),
                            R(6) * (W0 + R(4) * W1 - R(5) * W2 + R(4) * s1 + R(2) * s2));
  // linear weights d^6_k / d^8_k (Sec. 3.3)
  R d0, d1, d2, d3, d4, d5, d6;
  if (ORDER == 6) {
    d0 = R(33.0 / 700); d1 = R(11.0 / 140); d2 = R(22.0 / 175); d3 = R(11.0 / 100);
    d4 = R(11.0 / 100); d5 = R(37.0 / 140); d6 = R(37.0 / 140);
  } else {
    d0 = R(3.0 / 98); d1 = R(5.0 / 98); d2 = R(4.0 / 49); d3 = R(7.0 / 98);
    d4 = R(7.0 / 98); d5 = R(17.0 / 49); d6 = R(17.0 / 49);
  }
  // WENO-Z weights, Eqs. (WENO-Z-w) and (tau)
  R Z = fabs(R(3) * (c0.b - c4.b) + (c4.b - c3.b));
  R a0 = d0 * (R(1) + fdiv<R>(Z, c0.b + eps));
  R a1 = d1 * (R(1) + fdiv<R>(Z, b1 + eps));
  R a2 = d2 * (R(1) + fdiv<R>(Z, c2.b + eps));
  R a3 = d3 * (R(1) + fdiv<R>(Z, c3.b + eps));
  R a4 = d4 * (R(1) + fdiv<R>(Z, c4.b + eps));
  R a5 = d5 * (R(1) + fdiv<R>(Z, c5.b + eps));
  R a6 = d6 * (R(1) + fdiv<R>(Z, c6.b + eps));
  R inv = fdiv<R>(R(1), a0 + a1 + a2 + a3 + a4 + a5 + a6);
  // w_1 and w_3 share point value and slope
  val = (a0 * c0.v + (a1 + a3) * c3.v + a2 * c2.v + a4 * c4.v + a5 * c5.v + a6 * c6.v) * inv;
  dh = (a0 * c0.d + (a1 + a3) * c3.d + a2 * c2.d + a4 * c4.d + a5 * c5.d + a6 * c6.d) * inv;
}

// ---------------------------------------------------------------------------
// Characteristic projection (Sec. 3.1, characteristic variables) with the Euler
// eigenvectors of the interface-normal direction at state (rho, U, V, H, c).
// Right eigenvectors: (1, U-c, V, H-Uc), (1, U, V, q^2/2), (0, 0, 1, V), (1, U+c, V, H+Uc).
// ---------------------------------------------------------------------------
template <typename R, int DIM>
struct Eig {
  R U, V, H, c, b1, b2, ic;
};

template <typename R, int DIM>
__device__ __forceinline__ Eig<R, DIM> eig_at(const R* W, R gamma) {
  Eig<R, DIM> e;
  R irho = fdiv<R>(R(1), W[0]);
  e.U = W[1] * irho;
  e.V = DIM == 2 ? W[2] * irho : R(0);
  R q2 = e.U * e.U + e.V * e.V;
  R p = (gamma - R(1)) * (W[DIM + 1] - R(0.5) * W[0] * q2);
  R c2 = gamma * p * irho;
  e.c = fsqrt<R>(c2);
  e.ic = fdiv<R>(R(1), e.c);
  e.H = (W[DIM + 1] + p) * irho;
  e.b1 = fdiv<R>(gamma - R(1), c2);
  e.b2 = R(0.5) * q2 * e.b1;
  return e;
}

// w = L q (project conservative -> characteristic)
template <typename R, int DIM>
__device__ __forceinline__ void eig_left(const Eig<R, DIM>& e, const R* q, R* w) {
  const int N = DIM + 2;
  R E = q[N - 1];
  R mU = e.U * q[1] + (DIM == 2 ? e.V * q[2] : R(0));
  R base = e.b2 * q[0] - e.b1 * mU + e.b1 * E;   // b2 q0 - b1 (U q1 + V q2) + b1 E
  R acou = e.ic * (e.U * q[0] - q[1]);
  w[0] = R(0.5) * (base + acou);
  w[1] = q[0] - base;
  if (DIM == 2) w[2] = q[2] - e.V * q[0];
  w[N - 1] = R(0.5) * (base - acou);
}

// q = R w (back to conservative)
template <typename R, int DIM>
__device__ __forceinline__ void eig_right(const Eig<R, DIM>& e, const R* w, R* q) {
  const int N = DIM + 2;
  R wa = w[0], wb = w[1], wd = w[N - 1];
  R wc = DIM == 2 ? w[2] : R(0);
  q[0] = wa + wb + wd;
  q[1] = (e.U - e.c) * wa + e.U * wb + (e.U + e.c) * wd;
  if (DIM == 2) q[2] = e.V * (wa + wb + wd) + wc;
  q[N - 1] = (e.H - e.U * e.c) * wa + R(0.5) * (e.U * e.U + e.V * e.V) * wb + (e.H + e.U * e.c) * wd +
             (DIM == 2 ? e.V * wc : R(0));
}

// ---------------------------------------------------------------------------
// Maxwellian and its moments (Sec. 2.1).  g = rho (lam/pi)^{(K+DIM)/2} e^{-lam c^2}.
// m[k] = <u^k> (full or half space), n[k] = <v^k>, x1 = <xi^2>, x2 = <xi^4>.
// ---------------------------------------------------------------------------
template <typename R, int DIM>
struct Maxw {
  R rho, U, V, lam, p;
  R m[7];
  R n[7];
  R x1, x2;
  // constants of the closed-form moment solve
  R irho, Q, lam2, cK;
};

template <typename R, int DIM>
__device__ __forceinline__ bool maxw_prim(const R* W, R gamma, R K, Maxw<R, DIM>& g) {
  g.rho = W[0];
  const R irho = fdiv<R>(R(1), g.rho);
  g.U = W[1] * irho;
  g.V = DIM == 2 ? W[2] * irho : R(0);
  g.p = (gamma - R(1)) * (W[DIM + 1] - R(0.5) * g.rho * (g.U * g.U + g.V * g.V));
  g.lam = fdiv<R>(R(0.5) * g.rho, g.p);
  R h = g.p * irho;      // variance 1/(2 lam) = p / rho
  g.x1 = K * h;
  g.x2 = K * (K + R(2)) * h * h;
  g.irho = irho;
  g.Q = g.U * g.U + g.V * g.V + (K + R(DIM)) * h;
  g.lam2 = R(2) * g.lam;
  g.cK = fdiv<R>(g.lam2 * g.lam2, K + R(DIM));
  if (DIM == 2) {
    g.n[0] = R(1); g.n[1] = g.V;
#pragma unroll
    for (int k = 1; k < 6; ++k) g.n[k + 1] = g.V * g.n[k] + R(k) * h * g.n[k - 1];
  }
  return (g.rho > R(0)) && (g.p > R(0));
}

// full-space u moments
template <typename R, int DIM>
__device__ __forceinline__ void maxw_full(Maxw<R, DIM>& g) {
  R h = g.p * g.irho;
  g.m[0] = R(1); g.m[1] = g.U;
#pragma unroll
  for (int k = 1; k < 6; ++k) g.m[k + 1] = g.U * g.m[k] + R(k) * h * g.m[k - 1];
}

// half-space u moments: sign = +1 for u > 0, -1 for u < 0
template <typename R, int DIM>
__device__ __forceinline__ void maxw_half(Maxw<R, DIM>& g, int sign) {
  R h = g.p * g.irho;
  R sl = fsqrt<R>(g.lam);
  R s = sign > 0 ? R(1) : R(-1);
  g.m[0] = R(0.5) * erfc(-s * sl * g.U);
  g.m[1] = g.U * g.m[0] + fdiv<R>(s * R(0.5) * exp(-g.lam * g.U * g.U), sl * R(1.7724538509055160273));
#pragma unroll
  for (int k = 1; k < 6; ++k) g.m[k + 1] = g.U * g.m[k] + R(k) * h * g.m[k - 1];
}

// Closed-form solution of rho <psi (a.psi)> = b (verified symbolically against the moment
// matrix of the Maxwellian).
template <typename R, int DIM>
__device__ __forceinline__ void maxw_solve(const Maxw<R, DIM>& g, const R* b, R* a) {
  const R irho = g.irho, Q = g.Q, lam2 = g.lam2, cK = g.cK;
  R b1 = b[0] * irho, b2 = b[1] * irho;
  R R2 = b2 - g.U * b1;
  if (DIM == 2) {
    R b3 = b[2] * irho, b4 = b[3] * irho;
    R R3 = b3 - g.V * b1;
    R R4 = R(2) * b4 - Q * b1;
    R a4 = cK * (R4 - R(2) * g.U * R2 - R(2) * g.V * R3);
    R a3 = lam2 * R3 - g.V * a4;
    R a2 = lam2 * R2 - g.U * a4;
    a[0] = b1 - g.U * a2 - g.V * a3 - R(0.5) * a4 * Q;
    a[1] = a2; a[2] = a3; a[3] = a4;
  } else {
    R b3 = b[2] * irho;
    R R3 = R(2) * b3 - Q * b1;
    R a3 = cK * (R3 - R(2) * g.U * R2);
    R a2 = lam2 * R2 - g.U * a3;
    a[0] = b1 - g.U * a2 - R(0.5) * a3 * Q;
    a[1] = a2; a[2] = a3;
  }
}

// Symmetric moment operator G[k][l] = <psi_k psi_l u^A v^B> over the u-moments in m.
template <typename R, int DIM>
struct Gm { R e[DIM == 2 ? 10 : 6]; };

template <typename R, int DIM, int A, int B>
__device__ __forceinline__ Gm<R, DIM> gmat(const Maxw<R, DIM>& g) {
  Gm<R, DIM> G;
  const R* m = g.m;
  if (DIM == 2) {
    const R* n = g.n;
    auto E = [&](int p, int q) { return m[p] * n[q]; };
    R x1 = g.x1, x2 = g.x2;
    G.e[0] = E(A, B);                                                             // 00
    G.e[1] = E(A + 1, B);                                                         // 01
    G.e[2] = E(A, B + 1);                                                         // 02
    G.e[3] = R(0.5) * (E(A + 2, B) + E(A, B + 2) + E(A, B) * x1);                 // 03
    G.e[4] = E(A + 2, B);                                                         // 11
    G.e[5] = E(A + 1, B + 1);                                                     // 12
    G.e[6] = R(0.5) * (E(A + 3, B) + E(A + 1, B + 2) + E(A + 1, B) * x1);         // 13
    G.e[7] = E(A, B + 2);                                                         // 22
    G.e[8] = R(0.5) * (E(A + 2, B + 1) + E(A, B + 3) + E(A, B + 1) * x1);         // 23
    G.e[9] = R(0.25) * (E(A + 4, B) + E(A, B + 4) + E(A, B) * x2 +
                        R(2) * (E(A + 2, B + 2) + (E(A + 2, B) + E(A, B + 2)) * x1));  // 33
  } else {
    R x1 = g.x1, x2 = g.x2;
    G.e[0] = m[A];
    G.e[1] = m[A + 1];
    G.e[2] = R(0.5) * (m[A + 2] + m[A] * x1);
    G.e[3] = m[A + 2];
    G.e[4] = R(0.5) * (m[A + 3] + m[A + 1] * x1);
    G.e[5] = R(0.25) * (m[A + 4] + R(2) * m[A + 2] * x1 + m[A] * x2);
  }
  return G;
}

// out = s * G c  (+= if ACC)
template <typename R, int DIM, bool ACC>
__device__ __forceinline__ void gmul(const Gm<R, DIM>& G, const R* c, R s, R* out) {
  if (DIM == 2) {
    R o0 = G.e[0] * c[0] + G.e[1] * c[1] + G.e[2] * c[2] + G.e[3] * c[3];
    R o1 = G.e[1] * c[0] + G.e[4] * c[1] + G.e[5] * c[2] + G.e[6] * c[3];
    R o2 = G.e[2] * c[0] + G.e[5] * c[1] + G.e[7] * c[2] + G.e[8] * c[3];
    R o3 = G.e[3] * c[0] + G.e[6] * c[1] + G.e[8] * c[2] + G.e[9] * c[3];
    if (ACC) { out[0] += s * o0; out[1] += s * o1; out[2] += s * o2; out[3] += s * o3; }
    else { out[0] = s * o0; out[1] = s * o1; out[2] = s * o2; out[3] = s * o3; }
  } else {
    R o0 = G.e[0] * c[0] + G.e[1] * c[1] + G.e[2] * c[2];
    R o1 = G.e[1] * c[0] + G.e[3] * c[1] + G.e[4] * c[2];
    R o2 = G.e[2] * c[0] + G.e[4] * c[1] + G.e[5] * c[2];
    if (ACC) { out[0] += s * o0; out[1] += s * o1; out[2] += s * o2; }
    else { out[0] = s * o0; out[1] = s * o1; out[2] = s * o2; }
  }
}

// column 0 of G (moments <psi u^A v^B>)
template <typename R, int DIM>
__device__ __forceinline__ void gcol0(const Gm<R, DIM>& G, R s, R* out, bool acc) {
  if (DIM == 2) {
    R o[4] = {G.e[0], G.e[1], G.e[2], G.e[3]};
    for (int k = 0; k < 4; ++k) out[k] = acc ? out[k] + s * o[k] : s * o[k];
  } else {
    R o[3] = {G.e[0], G.e[1], G.e[2]};
    for (int k = 0; k < 3; ++k) out[k] = acc ? out[k] + s * o[k] : s * o[k];
  }
}

// ---------------------------------------------------------------------------
// FP64 time-integration coefficients of the exponential (non-equilibrium) terms.
// With E0(d) = int_0^d e^{-t/tau} dt, E1(d) = int_0^d t e^{-t/tau} dt and h = dt/2:
//   a0 = (4 E0(h) - E0(2h))/dt,      a1 = (4 E1(h) - E1(2h))/dt,
//   b0 = 4 (E0(2h) - 2 E0(h))/dt^2,  b1 = 4 (E1(2h) - 2 E1(h))/dt^2.
// These are the flux and flux-derivative weights of the linear-in-time fit over
// [0, dt/2] and [0, dt].  They cancel catastrophically when dt/tau is small, so they are
// evaluated from stable closed forms (x = h/tau, S = 1 - e^{-x} = -expm1(-x)):
//   4E0(h)-E0(2h) = tau S (2 + S),  E0(2h)-2E0(h) = -tau S^2,
// and for the E1 pair by their Taylor series in x when x < 1.
// ---------------------------------------------------------------------------
struct TimeCoef { double a0, a1, b0, b1; };

// Taylor coefficients of 4 phi(x) - phi(2x) and phi(2x) - 2 phi(x) for
// phi(y) = 1 - e^{-y}(1 + y) = sum_{k>=2} (-1)^k (k-1) y^k / k!, k = 2..21, and of
// S(x) = 1 - e^{-x} = sum_{k>=1} (-1)^(k+1) x^k / k!, formed at compile time.  The series are
// used for x < 1/2, where the first omitted term (of the truncation time_coefs picks for the
// range of x) is below 1e-19 of the terms' magnitude
// |4 phi(x)| + |phi(2x)| (resp. |phi(2x)| + |2 phi(x)|; for S, of S itself); from x = 1/2 on,
// the closed form loses at most a few ulp of that magnitude to cancellation (1e-15 measured
// against an 80-digit evaluation; at x -> 1 the series would leave 6e-14).
struct PhiSeries { double a[22], b[22], s[22]; };
__host__ __device__ constexpr PhiSeries make_phi_series() {
  PhiSeries c{};
  double fact = 1.0, p2 = 1.0;
  for (int k = 0; k < 22; ++k) {
    if (k > 0) { fact *= k; p2 *= 2.0; }
    const double sg = (k & 1) ? -1.0 : 1.0;
    c.a[k] = k >= 2 ? sg * (k - 1) * (4.0 - p2) / fact : 0.0;
    c.b[k] = k >= 2 ? sg * (k - 1) * (p2 - 2.0) / fact : 0.0;
    c.s[k] = k >= 1 ? -sg / fact : 0.0;
  }
  return c;
}

// sum_{j=0..M} c[OFF + j] x^j by Horner's rule in y = x^2 on the even and the odd
// coefficients separately, E(y) + x O(y): two independent chains of half the length, so the
// dependent FP64 latency per polynomial is halved for one extra operation.
template <int OFF, int M>
__device__ __forceinline__ double poly_even_odd(const double (&c)[22], double x, double y) {
  constexpr int ME = (M % 2 == 0) ? M : M - 1, MO = (M % 2 == 1) ? M : M - 1;
  double e = c[OFF + ME], o = c[OFF + MO];
#pragma unroll
  for (int j = ME - 2; j >= 0; j -= 2) e = fma(e, y, c[OFF + j]);
#pragma unroll
  for (int j = MO - 2; j >= 1; j -= 2) o = fma(o, y, c[OFF + j]);
  return fma(o, x, e);
}

// 4 phi(x) - phi(2x), phi(2x) - 2 phi(x) and 1 - e^{-x} by their series up to x^K.
template <int K>
__device__ __forceinline__ void time_series(double x, double& pa, double& pb, double& S) {
  constexpr PhiSeries C = make_phi_series();
  const double x2 = x * x;
  pa = poly_even_odd<2, K - 2>(C.a, x, x2) * x2;
  pb = poly_even_odd<2, K - 2>(C.b, x, x2) * x2;
  S = poly_even_odd<1, K - 1>(C.s, x, x2) * x;
}

// Arguments in terms of theta = tau/dt and x = (dt/2)/tau = 1/(2 theta) (both formed by the
// caller in its arithmetic type; the cancellation is inside the formulas below, which run in
// FP64): a0 = theta S (2 + S), b0 = -4 theta S^2 / dt, a1 = theta^2 dt pa, b1 = 4 theta^2 pb.
// SINGLE: the coefficients are rounded to float by the caller (the single-precision form),
// so the series stop where their truncation falls below 1e-9 of the result itself (k = 10,
// 11, 14 for x < 1/8, 1/4, 1/2; 3.4e-10 at most, measured with 50-digit arithmetic), far
// under the float rounding that follows; the arithmetic stays FP64 (the cancellation).
template <bool SINGLE = false>
__device__ __forceinline__ TimeCoef time_coefs(double theta, double x, double dt) {
  TimeCoef T;
  double S;        // 1 - e^{-x}
  double pa, pb;   // 4 phi(x) - phi(2x) and phi(2x) - 2 phi(x), phi(y) = 1 - e^{-y}(1+y)
  if (x < 0.5) {
    // the three series, by Horner's rule in x in lockstep (x^2, resp. x, factored out),
    // truncated after the last term that reaches 1e-19 of the magnitudes above: k = 15 for
    // x < 1/8, 17 for x < 1/4, 21 for x < 1/2 (fewer dependent FP64 steps for small x)
    if (x < 0.125) time_series<SINGLE ? 10 : 15>(x, pa, pb, S);
    else if (x < 0.25) time_series<SINGLE ? 11 : 17>(x, pa, pb, S);
    else time_series<SINGLE ? 14 : 21>(x, pa, pb, S);
  } else {
    // for x > 40, e^{-x} < 2^-57 and 1 - e^{-x} rounds to 1: S = 1 and e^{-x} = 0 exactly
    S = x > 40.0 ? 1.0 : -expm1(-x);
    double e = 1.0 - S;   // e^{-x}
    double e2 = e * e;
    pa = 3.0 - 4.0 * e * (1.0 + x) + e2 * (1.0 + 2.0 * x);
    pb = -1.0 + 2.0 * e * (1.0 + x) - e2 * (1.0 + 2.0 * x);
  }
  double idt = 1.0 / dt;
  T.a0 = theta * S * (2.0 + S);
  T.b0 = -4.0 * theta * S * S * idt;
  const double t2 = theta * theta;
  T.a1 = t2 * pa * dt;
  T.b1 = 4.0 * t2 * pb;
  return T;
}

// ---------------------------------------------------------------------------
// Gas-kinetic evaluation at one interface point (Eq. 3rd-simplify-flux, Sec. 2.2).
// ---------------------------------------------------------------------------
struct PhysParams {
  double gamma, K, mu, Pr, eps_tau, C_tau, weno_eps;
  float gammaf, Kf;   // single-precision copies of gamma and K (set with set_phys_floats)
  int tau_mode = 0;   // 0: bracket with mu/p (reading R1); 1: bracket with the numerical time
  int coef_mode = 0;  // equilibrium Taylor coefficients: 0 simplified (linearised chain); 1 full
                      // products (FP64 form, Euler; kernels instantiated with CM = true)
  int tan_mode = 0;   // 2D WENO-Z: 0 tangential quartic for every face quantity; 1 tangential
                      // WENO-Z for the non-equilibrium states (tan_weno)
};

inline void set_phys_floats(PhysParams& P) { P.gammaf = (float)P.gamma; P.Kf = (float)P.K; }

// gamma and K in the arithmetic type R
template <typename R> __device__ __forceinline__ R phys_gamma(const PhysParams& P);
template <> __device__ __forceinline__ double phys_gamma<double>(const PhysParams& P) { return P.gamma; }
template <> __device__ __forceinline__ float phys_gamma<float>(const PhysParams& P) { return P.gammaf; }
template <typename R> __device__ __forceinline__ R phys_K(const PhysParams& P);
template <> __device__ __forceinline__ double phys_K<double>(const PhysParams& P) { return P.K; }
template <> __device__ __forceinline__ float phys_K<float>(const PhysParams& P) { return P.Kf; }

template <typename R, int DIM>
struct PointIn {
  R W0[DIM + 2], W0x[DIM + 2], W0xx[DIM + 2];
  R W0y[DIM + 2], W0xy[DIM + 2], W0yy[DIM + 2];
  R Wl[DIM + 2], Wlx[DIM + 2], Wly[DIM + 2];
  R Wr[DIM + 2], Wrx[DIM + 2], Wry[DIM + 2];
};

template <typename R, int DIM>
struct PointOut {
  R F[DIM + 2], Ft[DIM + 2], W0[DIM + 2], Wt[DIM + 2], Wtt[DIM + 2];
};

// Heat flux q = 1/2 rho <a (a^2 + b^2 + xi^2) P> of P = u (cu.psi) + v (cv.psi) + (c0.psi)
// over g0, with a = u - U, b = v - V centred Gaussians of variance h = 1/(2 lam).
// Each c.psi is rewritten about (U, V) as k0 + ka a + kb b + k4/2 C2 (C2 = a^2+b^2+xi^2);
// only the parts odd in a and even in b survive the average.
template <typename R, int DIM>
__device__ __forceinline__ R heat_lin(const Maxw<R, DIM>& g, const R* cu, const R* cv, const R* c0) {
  R h = fdiv<R>(R(0.5), g.lam);
  R U = g.U, V = DIM == 2 ? g.V : R(0);
  R bb2 = DIM == 2 ? h : R(0);                 // <b^2>
  R bb4 = DIM == 2 ? R(3) * h * h : R(0);      // <b^4>
  R a2 = h, a4 = R(3) * h * h, a6 = R(15) * h * h * h;
  R xi2 = g.x1, xi4 = g.x2;
  R Ia2 = a4 + a2 * bb2 + a2 * xi2;                                           // <a^2 C2>
  R Ia2C4 = a6 + a2 * bb4 + a2 * xi4 + R(2) * (a4 * bb2 + a4 * xi2 + a2 * bb2 * xi2);  // <a^2 C2^2>
  auto ka_of = [&](const R* c) { return c[1] + c[DIM + 1] * U; };
  auto k0_of = [&](const R* c) {
    R c3 = DIM == 2 ? c[2] : R(0);
    return c[0] + c[1] * U + c3 * V + R(0.5) * c[DIM + 1] * (U * U + V * V);
  };
  R q = ka_of(c0) * Ia2;                                          // (c0.psi): ka a
  q += (U * ka_of(cu) + k0_of(cu)) * Ia2 + R(0.5) * cu[DIM + 1] * Ia2C4;   // (U + a)(cu.psi)
  if (DIM == 2) q += V * ka_of(cv) * Ia2;                         // (V + b)(cv.psi)
  return R(0.5) * g.rho * q;
}

// ---------------------------------------------------------------------------
// Euler flux and flux-Jacobian products of the equilibrium state.
// For a Maxwellian, the perturbations (a.psi) g span the tangent space of the Maxwellian
// family, so rho<u psi (a.psi)> = A(W) rho<psi (a.psi)> and rho<v psi (a.psi)> = B(W) rho<psi
// (a.psi)> exactly, with A, B the Jacobians of the Euler fluxes.  The equilibrium branch of
// Eq. (3rd-simplify-flux) and its compatibility chain are therefore evaluated with A and B
// (no moments needed).  Local frame: A is the face-normal Jacobian, B the tangential one.
// ---------------------------------------------------------------------------
template <typename R, int DIM>
struct Flow { R rho, irho, U, V, p, H, g1, q2h; };

template <typename R, int DIM>
__device__ __forceinline__ Flow<R, DIM> flow_of(const R* W, R gamma) {
  Flow<R, DIM> f;
  f.rho = W[0];
  f.irho = fdiv<R>(R(1), f.rho);
  f.U = W[1] * f.irho;
  f.V = DIM == 2 ? W[2] * f.irho : R(0);
  f.q2h = R(0.5) * (f.U * f.U + f.V * f.V);
  f.g1 = gamma - R(1);
  f.p = f.g1 * (W[DIM + 1] - f.rho * f.q2h);
  f.H = (W[DIM + 1] + f.p) * f.irho;
  return f;
}

// o = A w (normal Jacobian)
template <typename R, int DIM>
__device__ __forceinline__ void jac_n(const Flow<R, DIM>& f, const R* w, R* o) {
  if (DIM == 2) {
    R dp = f.g1 * (w[3] - f.U * w[1] - f.V * w[2] + f.q2h * w[0]);
    R du = w[1] - f.U * w[0];
    o[0] = w[1];
    o[1] = f.U * (w[1] + du) + dp;
    o[2] = f.V * du + f.U * w[2];
    o[3] = f.U * (w[3] + dp) + f.H * du;
  } else {
    R dp = f.g1 * (w[2] - f.U * w[1] + f.q2h * w[0]);
    R du = w[1] - f.U * w[0];
    o[0] = w[1];
    o[1] = f.U * (w[1] + du) + dp;
    o[2] = f.U * (w[2] + dp) + f.H * du;
  }
}

// o = B w (tangential Jacobian, 2D)
template <typename R>
__device__ __forceinline__ void jac_t(const Flow<R, 2>& f, const R* w, R* o) {
  R dp = f.g1 * (w[3] - f.U * w[1] - f.V * w[2] + f.q2h * w[0]);
  R dv = w[2] - f.V * w[0];
  o[0] = w[2];
  o[1] = f.U * dv + f.V * w[1];
  o[2] = f.V * (w[2] + dv) + dp;
  o[3] = f.V * (w[3] + dp) + f.H * dv;
}

// o = -(A x + B y)  (B term only in 2D)
template <typename R, int DIM>
__device__ __forceinline__ void neg_div(const Flow<R, DIM>& f, const R* x, const R* y, R* o) {
  const int N = DIM + 2;
  R a[N];
  jac_n<R, DIM>(f, x, a);
  if (DIM == 2) {
    R b[4];
    jac_t<R>(*reinterpret_cast<const Flow<R, 2>*>(&f), y, b);
#pragma unroll
    for (int k = 0; k < N; ++k) o[k] = -(a[k] + b[k]);
  } else {
#pragma unroll
    for (int k = 0; k < N; ++k) o[k] = -a[k];
  }
}

// Second derivatives of the Euler fluxes contracted with two perturbations u, v of the
// conservative variables: oF = (dA/dW . u) v for the normal flux, oG = (dB/dW . u) v for the
// tangential one (2D), from the flux components m U + p, n U, (E + p) U (normal) and m V,
// n V + p, (E + p) V (tangential) with U = m / rho, V = n / rho and
// p = (gamma - 1)(E - (m^2 + n^2) / (2 rho)):
//   d2U[u, v] = -(u_rho dU[v] + v_rho dU[u]) / rho,   d2p[u, v] = -(gamma - 1) rho (dU[u] dU[v] + dV[u] dV[v]).
template <typename R, int DIM>
__device__ __forceinline__ void euler_hess(const Flow<R, DIM>& f, const R* u, const R* v, R* oF, R* oG) {
  const int N = DIM + 2;
  const R uU = (u[1] - f.U * u[0]) * f.irho, vU = (v[1] - f.U * v[0]) * f.irho;
  const R uV = DIM == 2 ? (u[2] - f.V * u[0]) * f.irho : R(0), vV = DIM == 2 ? (v[2] - f.V * v[0]) * f.irho : R(0);
  const R up = f.g1 * (u[N - 1] - f.U * u[1] - (DIM == 2 ? f.V * u[2] : R(0)) + f.q2h * u[0]);
  const R vp = f.g1 * (v[N - 1] - f.U * v[1] - (DIM == 2 ? f.V * v[2] : R(0)) + f.q2h * v[0]);
  const R d2U = -(u[0] * vU + v[0] * uU) * f.irho;
  const R d2V = DIM == 2 ? -(u[0] * vV + v[0] * uV) * f.irho : R(0);
  const R d2p = -f.g1 * f.rho * (uU * vU + uV * vV);
  const R m = f.rho * f.U, n = f.rho * f.V, Ep = f.rho * f.H;
  oF[0] = R(0);
  oF[1] = u[1] * vU + v[1] * uU + m * d2U + d2p;
  if (DIM == 2) oF[2] = u[2] * vU + v[2] * uU + n * d2U;
  oF[N - 1] = (u[N - 1] + up) * vU + (v[N - 1] + vp) * uU + Ep * d2U + f.U * d2p;
  if (DIM == 2) {
    oG[0] = R(0);
    oG[1] = u[1] * vV + v[1] * uV + m * d2V;
    oG[2] = u[2] * vV + v[2] * uV + n * d2V + d2p;
    oG[3] = (u[3] + up) * vV + (v[3] + vp) * uV + Ep * d2V + f.V * d2p;
  }
}

// Change of the Euler flux (normal direction) between the reference state r and r + d,
// F(r + d) - F(r), written so that every term is a product with a component of d: in
// single precision its error is relative to the change, not to the flux.
template <typename R, int DIM>
__device__ __forceinline__ void euler_flux_delta(const R* r, const R* d, R gamma, R* o) {
  const int N = DIM + 2;
  R rho = r[0], m = r[1], n = DIM == 2 ? r[2] : R(0), E = r[N - 1];
  R drho = d[0], dm = d[1], dn = DIM == 2 ? d[2] : R(0), dE = d[N - 1];
  R irho = fdiv<R>(R(1), rho);
  R q = fdiv<R>(irho, rho + drho);                             // 1 / (rho (rho + drho))
  R U = m * irho, V = n * irho;
  R dmm = (rho * dm * (R(2) * m + dm) - m * m * drho) * q;    // d(m^2/rho)
  R dnn = (rho * dn * (R(2) * n + dn) - n * n * drho) * q;    // d(n^2/rho)
  R dU = (rho * dm - m * drho) * q;                           // d(m/rho)
  R p = (gamma - R(1)) * (E - R(0.5) * (m * U + n * V));
  R dp = (gamma - R(1)) * (dE - R(0.5) * (dmm + dnn));
  o[0] = dm;
  o[1] = dmm + dp;
  if (DIM == 2) o[2] = (rho * (m * dn + n * dm + dm * dn) - m * n * drho) * q;   // d(mn/rho)
  o[N - 1] = (E + p) * dU + (dE + dp) * (U + dU);
}

// DELTA: single-precision form.  in.W0, in.Wl, in.Wr hold full states ref + delta (used by
// the nonlinear functions), d0 the delta of the linear reconstruction value; out.F is then
// F - F_Euler(ref) and out.W0 is W0 - ref (the FP64 reference parts are added in the cell
// update).
// NEED_F = false (used by the second MSMD stage, which needs only F_t and W_tt): the flux and
// interface-value outputs F, W0 and the flux half of the bracket and of the non-equilibrium
// branch are not computed (out.F = out.W0 = 0).
// CM: the full-product equilibrium coefficients (coef_mode 1; Euler only, VISC false): the
// chain below gains the Euler fluxes' second-derivative terms.
template <typename R, int DIM, bool WENO, bool VISC, bool DELTA = false, bool NEED_F = true, bool CM = false>
__device__ __forceinline__ bool gks_point(const PhysParams& P, const PointIn<R, DIM>& in, double dt,
                                          PointOut<R, DIM>& out, const R* ref = nullptr,
                                          const R* d0 = nullptr) {
  const int N = DIM + 2;
  const R gamma = phys_gamma<R>(P), K = phys_K<R>(P);
  bool ok = true;
  R W0c[N];
  R pl = R(0), pr = R(0);
  if (WENO) {
    // Equilibrium value from the collision of the two initial states:
    // W0 = int_{u>0} psi g_l + int_{u<0} psi g_r.
    Maxw<R, DIM> gl, gr;
    ok &= maxw_prim<R, DIM>(in.Wl, gamma, K, gl);
    ok &= maxw_prim<R, DIM>(in.Wr, gamma, K, gr);
    maxw_half<R, DIM>(gl, +1);
    maxw_half<R, DIM>(gr, -1);
    Gm<R, DIM> Gl = gmat<R, DIM, 0, 0>(gl), Gr = gmat<R, DIM, 0, 0>(gr);
    gcol0<R, DIM>(Gl, gl.rho, W0c, false);
    gcol0<R, DIM>(Gr, gr.rho, W0c, true);
    pl = gl.p; pr = gr.p;
  } else {
#pragma unroll
    for (int k = 0; k < N; ++k) W0c[k] = in.W0[k];
  }
  const Flow<R, DIM> f = flow_of<R, DIM>(W0c, gamma);
  ok &= (f.rho > R(0)) && (f.p > R(0));

  // Equilibrium branch at t = 0 (readings R4-R6): F = F_Euler(W0), W_t = -(A W_x + B W_y),
  // W_xt = -(A W_xx + B W_xy), W_yt = -(A W_xy + B W_yy), W_tt = -(A W_xt + B W_yt), F_t = A W_t.
  R F[N], Ft[N], Wt[N], Wxt[N], Wyt[N], Wtt[N];
  R dW0[N];   // W0 - ref in the DELTA form
  if (!NEED_F) {
#pragma unroll
    for (int k = 0; k < N; ++k) { F[k] = R(0); dW0[k] = R(0); }
  } else if (DELTA) {
#pragma unroll
    for (int k = 0; k < N; ++k) dW0[k] = WENO ? W0c[k] - ref[k] : d0[k];
    euler_flux_delta<R, DIM>(ref, dW0, gamma, F);
  } else {
    R m = W0c[1];
    F[0] = m;
    F[1] = m * f.U + f.p;
    if (DIM == 2) F[2] = m * f.V;
    F[N - 1] = f.U * (W0c[N - 1] + f.p);
  }
  neg_div<R, DIM>(f, in.W0x, in.W0y, Wt);
  neg_div<R, DIM>(f, in.W0xx, in.W0xy, Wxt);
  if (DIM == 2) neg_div<R, DIM>(f, in.W0xy, in.W0yy, Wyt);
  if constexpr (CM) {
    // the Cauchy-Kowalewski derivatives of the Euler equations:
    // W_xt = -(A W_xx + B W_xy + A'[W_x] W_x + B'[W_x] W_y), W_yt likewise
    static_assert(!VISC, "the full-product coefficients are defined without the bracket");
    R hF[N], hG[N];
    euler_hess<R, DIM>(f, in.W0x, in.W0x, hF, hG);
#pragma unroll
    for (int k = 0; k < N; ++k) Wxt[k] -= hF[k];
    if (DIM == 2) {
      // A'[W_y] W_x = A'[W_x] W_y (the Hessian is symmetric)
      R hyF[N], hyG[N];
      euler_hess<R, DIM>(f, in.W0x, in.W0y, hF, hG);
      euler_hess<R, DIM>(f, in.W0y, in.W0y, hyF, hyG);
#pragma unroll
      for (int k = 0; k < N; ++k) { Wxt[k] -= hG[k]; Wyt[k] -= hF[k] + hyG[k]; }
    }
  }
  neg_div<R, DIM>(f, Wxt, Wyt, Wtt);
  if constexpr (CM) {   // W_tt = -(A W_xt + B W_yt + A'[W_t] W_x + B'[W_t] W_y)
    R hF[N], hG[N];
    euler_hess<R, DIM>(f, Wt, in.W0x, hF, hG);
#pragma unroll
    for (int k = 0; k < N; ++k) Wtt[k] -= hF[k];
    if (DIM == 2) {
      euler_hess<R, DIM>(f, Wt, in.W0y, hF, hG);
#pragma unroll
      for (int k = 0; k < N; ++k) Wtt[k] -= hG[k];
    }
  }
  jac_n<R, DIM>(f, Wt, Ft);

  if (VISC || WENO) {
    Maxw<R, DIM> g0;
    maxw_prim<R, DIM>(W0c, gamma, K, g0);
    maxw_full<R, DIM>(g0);
    const R rho0 = g0.rho;
    R a1[N], a2[N];
    maxw_solve<R, DIM>(g0, in.W0x, a1);
    if (DIM == 2) maxw_solve<R, DIM>(g0, in.W0y, a2);
    Gm<R, DIM> G20 = gmat<R, DIM, 2, 0>(g0);
    Gm<R, DIM> G11;
    if (DIM == 2) G11 = gmat<R, DIM, 1, 1>(g0);
    if (VISC) {
      // Chapman-Enskog bracket with the physical collision time mu/p (reading R1):
      // -tau rho<u psi (a1 u + a2 v + A)> and -tau rho<u psi (a_xt u + a_yt v + a_tt)>,
      // where rho<u psi A> = A_n W_t = F_t and rho<u psi a_tt> = A_n W_tt.
      // tau_mode 1 takes the numerical time of Sec. 4 instead: mu/p, or eps dt for the Euler
      // equations, plus C |pl - pr| / (pl + pr) dt (zero for the linear reconstruction,
      // whose two sides are one state).
      R tau = fdiv<R>(R(P.mu), g0.p);
      if (P.tau_mode == 1) {
        if (!(P.mu > 0.0)) tau = R(P.eps_tau) * R(dt);
        if (WENO) tau += R(P.C_tau) * fabs(fdiv<R>(pl - pr, pl + pr)) * R(dt);
      }
      R A[N], axt[N], ayt[N], att[N], Fvt[N];
      if (NEED_F) maxw_solve<R, DIM>(g0, Wt, A);
      maxw_solve<R, DIM>(g0, Wxt, axt);
      maxw_solve<R, DIM>(g0, Wtt, att);
      if (DIM == 2) maxw_solve<R, DIM>(g0, Wyt, ayt);
      jac_n<R, DIM>(f, Wtt, Fvt);
      R Fb[N], Fbt[N];
      if (NEED_F) gmul<R, DIM, false>(G20, a1, rho0, Fb);
      gmul<R, DIM, false>(G20, axt, rho0, Fbt);
      if (DIM == 2) {
        if (NEED_F) gmul<R, DIM, true>(G11, a2, rho0, Fb);
        gmul<R, DIM, true>(G11, ayt, rho0, Fbt);
      }
#pragma unroll
      for (int k = 0; k < N; ++k) {
        if (NEED_F) F[k] += -tau * (Fb[k] + Ft[k]);
        Ft[k] += -tau * (Fbt[k] + Fvt[k]);
      }
      if (P.Pr != 1.0) {
        // Prandtl-number fix (reading R10): (1/Pr - 1) q of the bracket terms.
        R fpr = R(1.0 / P.Pr - 1.0);
        if (NEED_F) F[N - 1] += fpr * (-tau * heat_lin<R, DIM>(g0, a1, a2, A));
        Ft[N - 1] += fpr * (-tau * heat_lin<R, DIM>(g0, axt, ayt, att));
      }
    }
    if (WENO) {
      // Non-equilibrium branch: -e^{-t/tau} g0 [1 - (a1 u + a2 v) t] + H g_l [...] + (1-H) g_r [...]
      // time-integrated over [0, dt/2] and [0, dt] and fitted linearly (FP64 coefficients).
      // rho0 <u psi> = F_Euler(W0).
      // theta = tau_n / dt (Sec. 4: mu/p, or eps dt, plus C |pl - pr| / (pl + pr) dt)
      const R theta = (P.mu > 0.0 ? fdiv<R>(R(P.mu), g0.p * R(dt)) : R(P.eps_tau)) +
                      R(P.C_tau) * fabs(fdiv<R>(pl - pr, pl + pr));
      const TimeCoef T = time_coefs<sizeof(R) == 4>((double)theta, (double)fdiv<R>(R(0.5), theta), dt);
      // c0 starts from minus the collisionless flux of g0 (F_Euler(W0); the bracket is not
      // part of it), formed here so that it does not depend on F being computed
      R c0[N], c1[N];
      {
        R m = W0c[1];
        c0[0] = -m; c0[1] = -(m * f.U + f.p);
        if (DIM == 2) c0[2] = -m * f.V;
        c0[N - 1] = -f.U * (W0c[N - 1] + f.p);
      }
      gmul<R, DIM, false>(G20, a1, rho0, c1);
      if (DIM == 2) gmul<R, DIM, true>(G11, a2, rho0, c1);
#pragma unroll
      for (int side = 0; side < 2; ++side) {
        Maxw<R, DIM> gk;
        R ak1[N], ak2[N];
        ok &= maxw_prim<R, DIM>(side == 0 ? in.Wl : in.Wr, gamma, K, gk);
        maxw_half<R, DIM>(gk, side == 0 ? +1 : -1);
        Gm<R, DIM> H10 = gmat<R, DIM, 1, 0>(gk);
        gcol0<R, DIM>(H10, gk.rho, c0, true);
        maxw_solve<R, DIM>(gk, side == 0 ? in.Wlx : in.Wrx, ak1);
        Gm<R, DIM> H20 = gmat<R, DIM, 2, 0>(gk);
        gmul<R, DIM, true>(H20, ak1, -gk.rho, c1);
        if (DIM == 2) {
          maxw_solve<R, DIM>(gk, side == 0 ? in.Wly : in.Wry, ak2);
          Gm<R, DIM> H11 = gmat<R, DIM, 1, 1>(gk);
          gmul<R, DIM, true>(H11, ak2, -gk.rho, c1);
        }
      }
      // the coefficients in the arithmetic type (FP64 for the FP64 form; rounded once to float
      // for the single-precision form, whose inputs c0, c1, F carry single-precision error)
      const R a0 = R(T.a0), a1 = R(T.a1), b0 = R(T.b0), b1 = R(T.b1);
#pragma unroll
      for (int k = 0; k < N; ++k) {
        if (NEED_F) F[k] = F[k] + a0 * c0[k] + a1 * c1[k];
        Ft[k] = Ft[k] + b0 * c0[k] + b1 * c1[k];
      }
    }
  }
#pragma unroll
  for (int k = 0; k < N; ++k) {
    out.F[k] = F[k]; out.Ft[k] = Ft[k];
    out.W0[k] = DELTA ? dW0[k] : W0c[k]; out.Wt[k] = Wt[k]; out.Wtt[k] = Wtt[k];
  }
  return ok;
}

}  // namespace gks
