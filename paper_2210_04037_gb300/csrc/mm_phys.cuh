// Device-side closures, mixture rule, fluxes and Riemann solver of the
// diffuse-interface elastoplastic method (Wallis, Barton & Nikiforakis,
// arXiv 2210.04037), templated on the precision policy:
//   P64: every quantity in FP64; the deformation tensor is carried as Fbar
//        and every closure is evaluated in the order of its definition, so
//        the only differences from a plain FP64 evaluation are the last-ulp
//        differences of the math library.
//   P32: reconstruction, fluxes and closures in FP32; total energy, the
//        energy recovery, the plastic-return iteration and all totals in
//        FP64.  The deformation tensor is carried as A = Fbar - I so that the
//        small elastic strains of metals keep their relative precision.
#pragma once

#include <math.h>
#include <stdint.h>

#include "mm_internal.h"

namespace mm {

typedef double E;  // energy scalar type in both precisions

// R: working precision; S: storage of the R fields; X: the second block
// (rho E / p and the volume fractions); allphi: all N volume fractions are
// carried (each its own advected field) instead of N-1 with the last one
// 1 - sum, so no fraction is ever formed by cancellation.
struct P64 {
  typedef double R;
  typedef double S;
  typedef double X;
  static constexpr bool split = false;
  static constexpr bool aform = false;
  static constexpr bool allphi = false;
};
struct P32 {
  typedef float R;
  typedef float S;
  typedef float X;
  static constexpr bool split = true;
  static constexpr bool aform = true;
  static constexpr bool allphi = true;
};
// The same for grids holding a void material (eos 2: the void volume
// fraction of Sec. 2.1): the closures leave it out of the mass, the energy
// and the pressure equilibrium, and the sweeps open void at critically
// damaged faces in tension (Sec. 3.1).  Grids without void keep the plain
// policies (voidable false), whose kernels carry none of this.
struct P64V : P64 {
  static constexpr bool voidable = true;
};
struct P32V : P32 {
  static constexpr bool voidable = true;
};
template <class P, class = void> struct Voidable { static constexpr bool value = false; };
template <class P> struct Voidable<P, decltype((void)P::voidable)> {
  static constexpr bool value = P::voidable;
};

// ---------------------------------------------------------------- math ----
__device__ __forceinline__ double mlog(double x) { return log(x); }
__device__ __forceinline__ float mlog(float x) { return logf(x); }
__device__ __forceinline__ double mlog1p(double x) { return log1p(x); }
__device__ __forceinline__ float mlog1p(float x) { return log1pf(x); }
__device__ __forceinline__ double mexp(double x) { return exp(x); }
__device__ __forceinline__ float mexp(float x) { return expf(x); }
__device__ __forceinline__ double mexpm1(double x) { return expm1(x); }
__device__ __forceinline__ float mexpm1(float x) { return expm1f(x); }
__device__ __forceinline__ double msqrt(double x) { return sqrt(x); }
__device__ __forceinline__ float msqrt(float x) { return sqrtf(x); }
__device__ __forceinline__ double mpow(double x, double y) { return pow(x, y); }
// FP32 power by exp2(y log2 x) on the special-function unit (x > 0): the
// closures' powers of compression ratios need relative, not last-ulp, accuracy
__device__ __forceinline__ float mpow(float x, float y) { return exp2f(y * __log2f(x)); }
__device__ __forceinline__ double mcbrt(double x) { return cbrt(x); }
__device__ __forceinline__ float mcbrt(float x) { return cbrtf(x); }
__device__ __forceinline__ double mabs(double x) { return fabs(x); }
__device__ __forceinline__ float mabs(float x) { return fabsf(x); }
__device__ __forceinline__ bool mfinite(double x) { return isfinite(x); }
__device__ __forceinline__ bool mfinite(float x) { return isfinite(x); }

template <class R> struct Eps;
template <> struct Eps<double> {
  static constexpr double jacobi = 1e-32;
  static constexpr double unit = 2.220446049250313e-16;  // 2^-52
};
template <> struct Eps<float> {
  static constexpr float jacobi = 1e-14f;
  static constexpr float unit = 1.1920929e-07f;  // 2^-23
};

// -------------------------------------------------------------- layout ----
template <int DIM> struct FC;
template <> struct FC<1> {
  static constexpr int n = 3;
  __host__ __device__ static constexpr int idx(int c) { return c == 0 ? 0 : (c == 1 ? 4 : 8); }
};
template <> struct FC<2> {
  static constexpr int n = 5;
  __host__ __device__ static constexpr int idx(int c) {
    return c == 0 ? 0 : (c == 1 ? 1 : (c == 2 ? 3 : (c == 3 ? 4 : 8)));
  }
};
template <> struct FC<3> {
  static constexpr int n = 9;
  __host__ __device__ static constexpr int idx(int c) { return c; }
};

template <int DIM, int NMAT, int NH>
struct Lay {
  static constexpr int NPHI = NMAT - 1;
  static constexpr int NFC = FC<DIM>::n;
  static constexpr int oPHI = 0;
  static constexpr int oARHO = NPHI;
  static constexpr int oMOM = oARHO + NMAT;
  static constexpr int oE = oMOM + DIM;
  static constexpr int oF = oE + 1;
  static constexpr int oH = oF + NFC;
  static constexpr int oX = oH + 2 * NH;
  static constexpr int NF = oX + DIM;
};

// ------------------------------------------------- single-material EOS ----
// Reference curve of material m at phasic density rho, damage factor psi and
// shear invariant J2: e_ref = e_c + e_s, p_ref = rho^2 de_ref/drho,
// dp_ref/drho and G.  Romenskii cold energy psi K0/(2 rho alpha^2)
// (eta^alpha - 1)^2, G = psi G0 eta^(beta+1), e_s = G J2 / rho, so
// p_c = psi K0/(2 alpha^2) (2 alpha q eta^alpha - q^2) with q = eta^alpha - 1
// and p_s = beta G J2.  Ideal gas: all zero.  Gam: the Grueneisen
// coefficient at rho and dlg = rho Gamma'(rho) / Gamma, which enters the
// isentropic sound speed (zero where Gamma is constant).
// Steinberg variant (shear_model 1, Sec. 2.1.2 and the U-Nb closure of
// Sec. 4.3): G = psi (G0 + Gp p_c0 u), p_c0 the undamaged cold pressure,
// u = eta^(-1/3), so p_s = rho^2 de_s/drho = J2 (rho G' - G) and
// dp_s/drho = J2 rho G'', from p_c0' = K0 E ((2a-1) E + 1 - a) / (a rho),
// p_c0'' = K0 E ((2a-1)^2 E - (a-1)^2) / (a rho^2) (E = eta^a),
// u' = -u / (3 rho), u'' = 4 u / (9 rho^2); Gamma = Gamma0 + Gamma1 u +
// Gamma2 eta^(-gamma_s).  G = G' = G'' = 0 where G0 + Gp p_c0 u <= 0.
template <class R>
__device__ __forceinline__ void thermo(const MatK& m, R rho, R psi, R J2, R& e, R& p,
                                       R& dp, R& G, R& Gam, R& dlg) {
  Gam = R(m.Gamma);
  dlg = R(0);
  if (m.eos != 1) {  // ideal gas or void
    e = R(0); p = R(0); dp = R(0); G = R(0);
    return;
  }
  const R a = R(m.alpha), rho0 = R(m.rho0), K0 = R(m.K0), bb = R(m.beta);
  const R eta = rho / rho0;
  const R ea = (m.alpha == 1.0) ? eta : mpow(eta, a);
  const R q = ea - R(1);
  const R ec = psi * K0 / (R(2) * rho * a * a) * (q * q);
  const R pc = psi * K0 / (R(2) * a * a) * (R(2) * a * q * ea - q * q);
  const R dpc = psi * K0 * mpow(eta, a - R(1)) * ((R(2) * a - R(1)) * ea + (R(1) - a)) / (a * rho0);
  if (m.shear_model == 1) {
    const R pc0 = K0 / (R(2) * a * a) * (R(2) * a * q * ea - q * q);
    const R pc1 = K0 * ea * ((R(2) * a - R(1)) * ea + (R(1) - a)) / (a * rho);
    const R pc2 = K0 * ea * ((R(2) * a - R(1)) * (R(2) * a - R(1)) * ea -
                             (a - R(1)) * (a - R(1))) / (a * rho * rho);
    const R u = mpow(eta, R(-1.0 / 3.0));
    const R qs = pc0 * u;
    const R q2 = u * (pc2 - R(2) * pc1 / (R(3) * rho) + R(4) * pc0 / (R(9) * rho * rho));
    const R q1 = u * (pc1 - pc0 / (R(3) * rho));
    // no shear stiffness where the form turns negative (strong tension)
    const bool pos = R(m.G0) + R(m.Gp) * qs > R(0);
    const R Gs = pos ? psi * (R(m.G0) + R(m.Gp) * qs) : R(0);
    const R dG = pos ? psi * R(m.Gp) * q1 : R(0), d2G = pos ? psi * R(m.Gp) * q2 : R(0);
    e = ec + Gs * J2 / rho;
    p = pc + J2 * (rho * dG - Gs);
    dp = dpc + J2 * rho * d2G;
    G = Gs;
    const R g2 = mpow(eta, -R(m.gamma_s));
    Gam = R(m.Gamma0) + R(m.Gamma1) * u + R(m.Gamma2) * g2;
    dlg = (-R(m.Gamma1) * u / R(3) - R(m.gamma_s) * R(m.Gamma2) * g2) / Gam;
    return;
  }
  const R Gs = psi * R(m.G0) * mpow(eta, bb + R(1));
  e = ec + Gs * J2 / rho;
  p = pc + bb * Gs * J2;
  dp = dpc + bb * (bb + R(1)) * Gs * J2 / rho;
  G = Gs;
}

// The same closure in FP32 from the FP32 constants: one reciprocal of rho,
// eta^(alpha-1) = eta^alpha / eta, and the precomputed K0/(2 alpha^2) and
// K0/(alpha rho0) in place of divisions.
__device__ __forceinline__ void thermo(const MatKf& m, float rho, float psi, float J2, float& e,
                                       float& p, float& dp, float& G, float& Gam, float& dlg) {
  Gam = m.Gamma;
  dlg = 0.f;
  if (m.eos != 1) {  // ideal gas or void
    e = 0.f; p = 0.f; dp = 0.f; G = 0.f;
    return;
  }
  const float a = m.alpha, bb = m.beta;
  const float ir = 1.f / rho;
  const float eta = rho * m.inv_rho0;
  const float ea = m.alpha_one ? eta : mpow(eta, a);
  const float q = ea - 1.f;
  const float k2 = psi * m.K0_2a2;
  const float ec = k2 * ir * (q * q);
  const float pc = k2 * (2.f * a * q * ea - q * q);
  const float dpc = psi * m.K0_arho0 * (ea * m.rho0 * ir) * ((2.f * a - 1.f) * ea + (1.f - a));
  if (m.shear_model == 1) {  // Steinberg, as in the FP64 closure
    const float pc0 = m.K0_2a2 * (2.f * a * q * ea - q * q);
    const float pc1 = m.K0 * ea * ((2.f * a - 1.f) * ea + (1.f - a)) * ir / a;
    const float pc2 = m.K0 * ea * ((2.f * a - 1.f) * (2.f * a - 1.f) * ea - (a - 1.f) * (a - 1.f)) *
                      (ir * ir) / a;
    const float u = mpow(eta, -1.f / 3.f);
    const float q1 = u * (pc1 - pc0 * ir * (1.f / 3.f));
    const float q2 = u * (pc2 - 2.f * pc1 * ir * (1.f / 3.f) + 4.f * pc0 * (ir * ir) * (1.f / 9.f));
    const float g0 = m.G0 + m.Gp * pc0 * u;
    const float gp = g0 > 0.f ? psi * m.Gp : 0.f;  // G = 0 where the form is negative
    const float Gs = g0 > 0.f ? psi * g0 : 0.f;
    e = ec + Gs * J2 * ir;
    p = pc + J2 * (rho * gp * q1 - Gs);
    dp = dpc + J2 * rho * gp * q2;
    G = Gs;
    const float g2 = mpow(eta, -m.gamma_s);
    Gam = m.Gamma0 + m.Gamma1 * u + m.Gamma2 * g2;
    dlg = (-m.Gamma1 * u * (1.f / 3.f) - m.gamma_s * m.Gamma2 * g2) / Gam;
    return;
  }
  const float Gs = psi * m.G0 * mpow(eta, bb + 1.f);
  const float gj = Gs * J2;
  e = ec + gj * ir;
  p = pc + bb * gj;
  dp = dpc + bb * (bb + 1.f) * gj * ir;
  G = Gs;
}

// Material constants in the precision of the arithmetic: MatK (FP64) or
// MatKf (FP32).
template <class R> struct MatSel;
template <> struct MatSel<double> {
  typedef MatK T;
  __device__ static __forceinline__ const MatK& get(const KArgs& a, int l) { return a.mat[l]; }
};
template <> struct MatSel<float> {
  typedef MatKf T;
  __device__ static __forceinline__ const MatKf& get(const KArgs& a, int l) { return a.matf[l]; }
};
template <class R>
__device__ __forceinline__ const typename MatSel<R>::T& matp(const KArgs& a, int l) {
  return MatSel<R>::get(a, l);
}

// ------------------------------------------- Hencky strain by Jacobi ----
// One symmetric Schur rotation of the (P,Q) plane.
template <int P, int Q, class R>
__device__ __forceinline__ void jrot(R a[9], R V[9]) {
  const R apq = a[3 * P + Q];
  if (apq == R(0)) return;
  const R app = a[3 * P + P], aqq = a[3 * Q + Q];
  const R theta = (aqq - app) / (R(2) * apq);
  R t = R(1) / (mabs(theta) + msqrt(theta * theta + R(1)));
  if (theta < R(0)) t = -t;
  const R c = R(1) / msqrt(t * t + R(1));
  const R s = t * c;
  constexpr int K = 3 - P - Q;
  a[3 * P + P] = app - t * apq;
  a[3 * Q + Q] = aqq + t * apq;
  a[3 * P + Q] = R(0);
  a[3 * Q + P] = R(0);
  const R akp = a[3 * K + P], akq = a[3 * K + Q];
  a[3 * K + P] = c * akp - s * akq;
  a[3 * P + K] = a[3 * K + P];
  a[3 * K + Q] = s * akp + c * akq;
  a[3 * Q + K] = a[3 * K + Q];
#pragma unroll
  for (int r = 0; r < 3; ++r) {
    const R vp = V[3 * r + P], vq = V[3 * r + Q];
    V[3 * r + P] = c * vp - s * vq;
    V[3 * r + Q] = s * vp + c * vq;
  }
}

// Cyclic Jacobi on a symmetric 3x3 matrix (destroyed): eigenvalues mu and
// eigenvectors in the columns of V.
template <class R>
__device__ __forceinline__ void jacobi(R a[9], R mu[3], R V[9]) {
#pragma unroll
  for (int k = 0; k < 9; ++k) V[k] = (k % 4 == 0) ? R(1) : R(0);
  for (int sweep = 0; sweep < 50; ++sweep) {
    const R off = a[1] * a[1] + a[2] * a[2] + a[5] * a[5];
    const R dd = a[0] * a[0] + a[4] * a[4] + a[8] * a[8];
    if (off <= Eps<R>::jacobi * dd) break;
    jrot<0, 1>(a, V);
    jrot<0, 2>(a, V);
    jrot<1, 2>(a, V);
  }
  mu[0] = a[0];
  mu[1] = a[4];
  mu[2] = a[8];
}

// dev(H) = dev(1/2 ln b), b = Fbar Fbar^T, with its deviatoric eigenvalues h
// and eigenvectors V.  X is Fbar (AF = false) or A = Fbar - I (AF = true,
// where b - I = A + A^T + A A^T and ln(1 + mu) keeps small strains exact).
// Returns false if b is not positive definite.
template <bool AF, class R>
__device__ __forceinline__ bool hencky(const R X[9], R devH[9], R h[3], R V[9]) {
  R B[9];
#pragma unroll
  for (int i = 0; i < 3; ++i)
#pragma unroll
    for (int j = i; j < 3; ++j) {
      R s = X[3 * i + 0] * X[3 * j + 0] + X[3 * i + 1] * X[3 * j + 1] + X[3 * i + 2] * X[3 * j + 2];
      if (AF) s = X[3 * i + j] + X[3 * j + i] + s;
      B[3 * i + j] = s;
      B[3 * j + i] = s;
    }
  R mu[3];
  jacobi(B, mu, V);
#pragma unroll
  for (int k = 0; k < 3; ++k) {
    if (AF) {
      if (!(mu[k] > R(-1)) || !mfinite(mu[k])) return false;
      h[k] = R(0.5) * mlog1p(mu[k]);
    } else {
      if (!(mu[k] > R(0)) || !mfinite(mu[k])) return false;
      h[k] = R(0.5) * mlog(mu[k]);
    }
  }
  const R tr = (h[0] + h[1] + h[2]) / R(3);
#pragma unroll
  for (int k = 0; k < 3; ++k) h[k] -= tr;
#pragma unroll
  for (int i = 0; i < 3; ++i)
#pragma unroll
    for (int j = 0; j < 3; ++j)
      devH[3 * i + j] = V[3 * i + 0] * h[0] * V[3 * j + 0] + V[3 * i + 1] * h[1] * V[3 * j + 1] +
                        V[3 * i + 2] * h[2] * V[3 * j + 2];
  return true;
}

// Product O = X Y of two symmetric 3x3 matrices that commute (functions of
// one matrix), so O is symmetric: the upper triangle is formed and mirrored.
template <class R>
__device__ __forceinline__ void sym_mul(const R X[9], const R Y[9], R O[9]) {
#pragma unroll
  for (int i = 0; i < 3; ++i)
#pragma unroll
    for (int j = i; j < 3; ++j) {
      const R v = X[3 * i + 0] * Y[0 + j] + X[3 * i + 1] * Y[3 + j] + X[3 * i + 2] * Y[6 + j];
      O[3 * i + j] = v;
      O[3 * j + i] = v;
    }
}

// ln(I + B) of a symmetric B with |B|_F <= 0.5 by the series of the inverse
// hyperbolic tangent: ln(I + B) = 2 artanh(Z) = 2 sum_k Z^(2k-1)/(2k-1) with
// Z = B (2I + B)^-1, a function of B whose eigenvalues z = b/(2 + b) obey
// |z| <= |B|_F/(2 - |B|_F) <= 1/3.  K odd terms in Horner form in Z^2; the
// truncation, below z^(2K)/(2K+1) relative, stays under 2e-8 for the
// thresholds below (FP32 accuracy).  Returns false (leaving L unset) beyond
// |B|_F = 0.5, where the caller takes the eigen-decomposition.
template <class R>
__device__ __forceinline__ bool log_series(const R B[9], R L[9]) {
  const R n2 = B[0] * B[0] + B[4] * B[4] + B[8] * B[8] + R(2) * (B[1] * B[1] + B[2] * B[2] + B[5] * B[5]);
  int K;
  if (n2 <= R(4e-4)) K = 2;         // |z| <= 0.0102: z^4/5 < 3e-9
  else if (n2 <= R(1e-2)) K = 3;    // |z| <= 0.0527: z^6/7 < 4e-9
  else if (n2 <= R(0.04)) K = 4;    // |z| <= 0.112: z^8/9 < 3e-9
  else if (n2 <= R(0.09)) K = 5;    // |z| <= 0.177: z^10/11 < 3e-9
  else if (n2 <= R(0.16)) K = 6;    // |z| <= 0.25: z^12/13 < 5e-9
  else if (n2 <= R(0.25)) K = 7;    // |z| <= 1/3: z^14/15 < 2e-8
  else return false;
  // C = 2I + B (eigenvalues in [1.5, 2.5]); C^-1 = adj(C)/det(C)
  const R c00 = R(2) + B[0], c11 = R(2) + B[4], c22 = R(2) + B[8];
  const R c01 = B[1], c02 = B[2], c12 = B[5];
  const R a00 = c11 * c22 - c12 * c12, a11 = c00 * c22 - c02 * c02, a22 = c00 * c11 - c01 * c01;
  const R a01 = c02 * c12 - c01 * c22, a02 = c01 * c12 - c02 * c11, a12 = c01 * c02 - c00 * c12;
  const R id = R(1) / (c00 * a00 + c01 * a01 + c02 * a02);
  const R Ci[9] = {a00 * id, a01 * id, a02 * id, a01 * id, a11 * id,
                   a12 * id, a02 * id, a12 * id, a22 * id};
  R Z[9], Z2[9], P[9];
  sym_mul(B, Ci, Z);
  sym_mul(Z, Z, Z2);
  // P <- I/(2K-1); P <- I/(2k-1) + Z^2 P for k = K-1 .. 1; L = 2 Z P
  const R cK = R(1) / R(2 * K - 1);
#pragma unroll
  for (int q = 0; q < 9; ++q) P[q] = (q % 4 == 0) ? cK : R(0);
  for (int k = K - 1; k >= 1; --k) {
    R T[9];
    sym_mul(Z2, P, T);
    const R ck = R(1) / R(2 * k - 1);
#pragma unroll
    for (int q = 0; q < 9; ++q) P[q] = T[q] + ((q % 4 == 0) ? ck : R(0));
  }
  sym_mul(Z, P, L);
#pragma unroll
  for (int q = 0; q < 9; ++q) L[q] *= R(2);
  return true;
}

// Large-strain fallback of hencky_fast: one out-of-line copy, so the rarely
// taken eigen-decomposition does not bloat every inlined call site.  Its
// operands travel by value (in registers), so the call sites keep no copy of
// the tensor in local memory for the branch they almost never take.
struct F9 { float v[9]; };
struct F10 { float v[9]; float ok; };
static __device__ __noinline__ F10 hencky_jacobi_f32(F9 A) {
  float h[3], V[9];
  F10 r;
  r.ok = hencky<true>(A.v, r.v, h, V) ? 1.f : 0.f;
  return r;
}

// dev(H) and J2 = tr(dev(H)^2) of A = Fbar - I, by the series while
// |Fbar Fbar^T - I|_F <= 0.5 (every metal state, and all but the most
// distorted gas), else by the eigen-decomposition.
template <class R>
__device__ __forceinline__ bool hencky_fast(const R A[9], R devH[9], R& J2) {
  R B[9];
#pragma unroll
  for (int i = 0; i < 3; ++i)
#pragma unroll
    for (int j = i; j < 3; ++j) {
      const R s = A[3 * i + j] + A[3 * j + i] +
                  (A[3 * i + 0] * A[3 * j + 0] + A[3 * i + 1] * A[3 * j + 1] + A[3 * i + 2] * A[3 * j + 2]);
      B[3 * i + j] = s;
      B[3 * j + i] = s;
    }
  R L[9];
  if (log_series(B, L)) {
    const R tr = (L[0] + L[4] + L[8]) / R(3);
#pragma unroll
    for (int q = 0; q < 9; ++q) devH[q] = R(0.5) * (L[q] - ((q % 4 == 0) ? tr : R(0)));
  } else {
    F9 a9;
#pragma unroll
    for (int q = 0; q < 9; ++q) a9.v[q] = A[q];
    const F10 r = hencky_jacobi_f32(a9);
    if (r.ok == 0.f) return false;
#pragma unroll
    for (int q = 0; q < 9; ++q) devH[q] = r.v[q];
  }
  J2 = R(0);
#pragma unroll
  for (int q = 0; q < 9; ++q) J2 += devH[q] * devH[q];
  return mfinite(J2);
}

// exp(X) - I of a symmetric X with |X|_F <= 0.06 by its power series
// (truncation below 1e-10 relative).
template <class R>
__device__ __forceinline__ void expm1_series(const R X[9], R M[9]) {
  constexpr int K = 6;
  // Horner: E = X (I + X/2 (I + X/3 (I + X/4 (I + X/5 (I + X/6)))))
  R P[9];
#pragma unroll
  for (int q = 0; q < 9; ++q) P[q] = (q % 4 == 0) ? R(1) : R(0);
#pragma unroll
  for (int k = K; k >= 1; --k) {
    R Q[9];
#pragma unroll
    for (int i = 0; i < 3; ++i)
#pragma unroll
      for (int j = 0; j < 3; ++j)
        Q[3 * i + j] = (X[3 * i + 0] * P[0 + j] + X[3 * i + 1] * P[3 + j] + X[3 * i + 2] * P[6 + j]) / R(k);
    if (k > 1) {
#pragma unroll
      for (int q = 0; q < 9; ++q) P[q] = Q[q] + ((q % 4 == 0) ? R(1) : R(0));
    } else {
#pragma unroll
      for (int q = 0; q < 9; ++q) M[q] = Q[q];
    }
  }
}

// hencky_fast of the FP32 closure as one out-of-line copy: every state
// conversion calls it (up to five per cell in a sweep), and the inlined
// copies made the sweep kernels large enough that warps stalled on
// instruction fetch; by value in registers, as the Jacobi fallback.
// Measured on the 256^3 cylinder: x sweep 3.77 -> 3.54 ms, y 3.72 -> 3.52,
// CFL 0.50 -> 0.44, sources 1.56 -> 1.39 (z 3.11 -> 3.19).
struct F11 { float v[9]; float j2; float ok; };
static __device__ __noinline__ F11 hencky_fast_f32(F9 A) {
  F11 r;
  r.ok = hencky_fast<float>(A.v, r.v, r.j2) ? 1.f : 0.f;
  return r;
}

// ------------------------------------------------------------ states ----
// Derived quantities of one state: velocity, the stress column d (sigma_kd,
// momentum flux and tangential tractions), the stress row d (sigma_dk, energy
// flux), density, longitudinal sound speed, mixture shear modulus.
template <class R>
struct Aux {
  R u[3];
  R sd[3];
  R sr[3];
  R rho, cL, G;
};

// A state is carried as two blocks: v[NF] in the working precision R, and
// x[NX] in FP64 with x[0] = rho E (conserved) or p (primitive) and
// x[1 + l] = phi_l (l < N-1).  The slots of v at those positions are unused.
// Keeping the volume fractions in FP64 makes the minority fraction
// 1 - sum(phi) exact in FP32-split storage.
template <class P, int DIM, int NMAT, int NH>
struct Phys {
  typedef typename P::R R;
  typedef typename P::X XT;
  typedef Lay<DIM, NMAT, NH> L;
  static constexpr int NF = L::NF;
  static constexpr int NPX = P::allphi ? NMAT : L::NPHI;  // fractions in the X block
  static constexpr int NX = 1 + NPX;
  static constexpr bool AF = P::aform;
  static constexpr bool VD = Voidable<P>::value;

  // Material l is the void (grids with a void material only).
  __device__ static __forceinline__ bool isvoid(const KArgs& a, int l) {
    return VD && l == a.void_l;
  }

  // Full 3x3 stored tensor (Fbar, or A = Fbar - I): inactive comps are 0 off
  // the diagonal (and the diagonal is always stored).
  __device__ static __forceinline__ void fullX(const R* c, R X[9]) {
#pragma unroll
    for (int k = 0; k < 9; ++k) X[k] = R(0);
#pragma unroll
    for (int k = 0; k < L::NFC; ++k) X[FC<DIM>::idx(k)] = c[L::oF + k];
  }

  // Value of Fbar_ij from a stored component.
  __device__ static __forceinline__ R Fv(int i, int j, R s) {
    return AF ? ((i == j ? R(1) : R(0)) + s) : s;
  }

  __device__ static __forceinline__ R damage_of(const KArgs& a, const R* w, int l) {
    R D = R(0);
#pragma unroll
    for (int h = 0; h < NH; ++h)
      if (h == a.hslot[l]) D = w[L::oH + 2 * h + 1];
    return D;
  }

  // Volume fractions of all N materials from the X block.
  __device__ static __forceinline__ void fractions(const XT* x, XT phi[NMAT]) {
    if constexpr (P::allphi) {
#pragma unroll
      for (int l = 0; l < NMAT; ++l) phi[l] = x[1 + l];
    } else {
      XT s = XT(0);
#pragma unroll
      for (int l = 0; l < NMAT - 1; ++l) {
        phi[l] = x[1 + l];
        s += phi[l];
      }
      phi[NMAT - 1] = XT(1) - s;
    }
  }

  // Mixture quantities of the isobaric Allaire closure with one deformation
  // tensor: per-material e_ref, p_ref, dp_ref, Gamma_l and 1/Gamma_l at the
  // phase density (constant but for the Steinberg closure) with
  // rho Gamma'/Gamma, and xi = sum phi_l/Gamma_l, G_mix = sum phi_l G_l.
  struct Mix {
    R e[NMAT], p[NMAT], dp[NMAT], ga[NMAT], gi[NMAT], dg[NMAT];
    R xi, Gm, J2;
    R devH[9];
  };

  __device__ static __forceinline__ bool mixture(const KArgs& a, const R phi[NMAT],
                                                 const R rho[NMAT], const R D[NMAT],
                                                 const R X[9], Mix& mx) {
    if constexpr (P::split) {
      F9 a9;
#pragma unroll
      for (int q = 0; q < 9; ++q) a9.v[q] = X[q];
      const F11 r = hencky_fast_f32(a9);
      if (r.ok == 0.f) return false;
#pragma unroll
      for (int q = 0; q < 9; ++q) mx.devH[q] = r.v[q];
      mx.J2 = r.j2;
    } else {
      R h[3], V[9];
      if (!hencky<AF>(X, mx.devH, h, V)) return false;
      mx.J2 = h[0] * h[0] + h[1] * h[1] + h[2] * h[2];
    }
    mx.xi = R(0);
    mx.Gm = R(0);
#pragma unroll
    for (int l = 0; l < NMAT; ++l) {
      const auto& m = matp<R>(a, l);
      const R psi = m.damage != 0 ? R(1) - D[l] : R(1);
      R G;
      thermo(m, rho[l], psi, mx.J2, mx.e[l], mx.p[l], mx.dp[l], G, mx.ga[l], mx.dg[l]);
      // 1/Gamma_l: the host's constant, or its value at rho_l (Steinberg)
      mx.gi[l] = m.shear_model == 1 ? R(1) / mx.ga[l] : R(m.xi);
      if (isvoid(a, l)) continue;  // no part in the pressure equilibrium
      if constexpr (P::split)
        mx.xi += phi[l] * mx.gi[l];
      else
        mx.xi += phi[l] / mx.ga[l];
      mx.Gm += phi[l] * G;
    }
    return true;
  }

  // sigma = -p I + 2 G_mix dev(H); c_L^2 = c^2 + 4/3 G_mix/rho with the
  // frozen mixture speed xi c^2 = sum y_l xi_l c_l^2,
  // c_l^2 = dp_ref,l + (Gamma_l + 1 + rho Gamma_l'/Gamma_l)(p - p_ref,l)/rho_l.
  template <int AX>
  __device__ static __forceinline__ bool finish(const KArgs& a, R p, const R rho[NMAT],
                                                const R arho[NMAT], const Mix& mx, Aux<R>& ax,
                                                R nu = R(0)) {
    // with void in the cell the materials fill 1 - nu of it: the pressure
    // part of the stress is theirs times that (the shear part is weighted by
    // the fractions already)
    const R pm = VD ? p * (R(1) - nu) : p;
#pragma unroll
    for (int k = 0; k < 3; ++k) {
      ax.sd[k] = (k == AX ? -pm : R(0)) + R(2) * mx.Gm * mx.devH[3 * k + AX];
      ax.sr[k] = (k == AX ? -pm : R(0)) + R(2) * mx.Gm * mx.devH[3 * AX + k];
    }
    R s = R(0);
#pragma unroll
    for (int l = 0; l < NMAT; ++l) {
      if (isvoid(a, l)) continue;
      const R Gam = mx.ga[l];
      const R cl2 = mx.dp[l] + (Gam + R(1) + mx.dg[l]) * (p - mx.p[l]) / rho[l];
      if constexpr (P::split)
        s += (arho[l] / ax.rho) * mx.gi[l] * cl2;
      else
        s += (arho[l] / ax.rho) * (R(1) / Gam) * cl2;
    }
    const R c2 = s / mx.xi;
    ax.G = mx.Gm;
    const R cL2 = c2 + (R(4) / R(3)) * mx.Gm / ax.rho;
    if (!(cL2 > R(0)) || !mfinite(cL2)) return false;
    ax.cL = msqrt(cL2);
    return true;
  }

  // primitive (w, wx) -> conserved (c, cx); the total energy is also
  // returned in FP64 (rhoE_out, may be null) for storage.
  template <int AX>
  __device__ static bool w2u(const KArgs& a, const R* w, const XT* wx, R* c, XT* cx, Aux<R>& ax,
                             double* rhoE_out = nullptr) {
    XT phid[NMAT];
    R phi[NMAT], rho[NMAT], arho[NMAT], D[NMAT];
    fractions(wx, phid);
    ax.rho = R(0);
#pragma unroll
    for (int l = 0; l < NMAT; ++l) {
      if (isvoid(a, l)) {  // no mass; its fraction may be zero
        if (!(phid[l] >= XT(0))) return false;
        phi[l] = R(phid[l]);
        rho[l] = R(0);
        arho[l] = R(0);
        D[l] = R(0);
        continue;
      }
      if (!(phid[l] > XT(0))) return false;
      phi[l] = R(phid[l]);
      rho[l] = w[L::oARHO + l];
      if (!(rho[l] > R(0))) return false;
      arho[l] = phi[l] * rho[l];
      ax.rho += arho[l];
      D[l] = damage_of(a, w, l);
    }
#pragma unroll
    for (int k = 0; k < 3; ++k) ax.u[k] = k < DIM ? w[L::oMOM + k] : R(0);
    const E pE = E(wx[0]);
    const R p = R(wx[0]);
    R X[9];
    fullX(w, X);
    Mix mx;
    if (!mixture(a, phi, rho, D, X, mx)) return false;
    E rhoe = 0.0, ke = 0.0;
    R ske = R(0);
    (void)ske;
    if constexpr (P::split) {
      // FP32: the face states need float accuracy only
      R re = R(0);
#pragma unroll
      for (int l = 0; l < NMAT; ++l)
        if (!isvoid(a, l)) re += arho[l] * mx.e[l] + phi[l] * mx.gi[l] * (p - mx.p[l]);
      const R kef = R(0.5) * ax.rho * (ax.u[0] * ax.u[0] + ax.u[1] * ax.u[1] + ax.u[2] * ax.u[2]);
      // the FP32 sum equals the FP64 sum rounded to FP32 (double rounding is
      // exact for one addition); the FP64 total is formed only when asked for
      ske = re + kef;
      if (rhoE_out) {
        rhoe = E(re);
        ke = E(kef);
      }
    } else {
#pragma unroll
      for (int l = 0; l < NMAT; ++l)
        if (!isvoid(a, l))
          rhoe += E(arho[l] * mx.e[l]) + E(phi[l]) * (pE - E(mx.p[l])) / E(mx.ga[l]);
      ke = 0.5 * E(ax.rho) *
           (E(ax.u[0]) * E(ax.u[0]) + E(ax.u[1]) * E(ax.u[1]) + E(ax.u[2]) * E(ax.u[2]));
    }
#pragma unroll
    for (int l = 0; l < NPX; ++l) cx[1 + l] = phid[l];
#pragma unroll
    for (int l = 0; l < NMAT - 1; ++l) c[L::oPHI + l] = R(0);
#pragma unroll
    for (int l = 0; l < NMAT; ++l) c[L::oARHO + l] = arho[l];
#pragma unroll
    for (int k = 0; k < DIM; ++k) c[L::oMOM + k] = ax.rho * ax.u[k];
    c[L::oE] = R(0);
    if constexpr (P::split)
      cx[0] = XT(ske);
    else
      cx[0] = XT(rhoe + ke);
    if (rhoE_out) *rhoE_out = rhoe + ke;
#pragma unroll
    for (int k = 0; k < L::NFC; ++k) c[L::oF + k] = w[L::oF + k];
    const R nu = VD && a.void_l >= 0 ? phi[VD ? a.void_l : 0] : R(0);
#pragma unroll
    for (int l = 0; l < NMAT; ++l) {
#pragma unroll
      for (int h = 0; h < NH; ++h)
        if (a.hslot[l] == h) {
          c[L::oH + 2 * h] = arho[l] * w[L::oH + 2 * h];
          c[L::oH + 2 * h + 1] = arho[l] * w[L::oH + 2 * h + 1];
        }
    }
#pragma unroll
    for (int k = 0; k < DIM; ++k) c[L::oX + k] = w[L::oX + k];
    return finish<AX>(a, p, rho, arho, mx, ax, nu);
  }

  // conserved (c, cx) -> primitive (w, wx), with
  // p = (rho e - sum_l phi_l rho_l e_ref,l + sum_l phi_l p_ref,l / Gamma_l) / xi.
  // rhoE_d (may be null): the cell's total energy in FP64 (stored state);
  // face states pass null and use cx[0].
  template <int AX>
  __device__ static bool u2w(const KArgs& a, const R* c, const XT* cx, R* w, XT* wx, Aux<R>& ax,
                             const double* rhoE_d = nullptr, Mix* mxo = nullptr) {
    XT phid[NMAT];
    R phi[NMAT], rho[NMAT], arho[NMAT], D[NMAT];
    fractions(cx, phid);
    ax.rho = R(0);
#pragma unroll
    for (int l = 0; l < NMAT; ++l) {
      arho[l] = c[L::oARHO + l];
      if (isvoid(a, l)) {
        if (!(phid[l] >= XT(0))) return false;
        phi[l] = R(phid[l]);
        rho[l] = R(0);
        continue;
      }
      if (!(phid[l] > XT(0)) || !(arho[l] > R(0))) return false;
      phi[l] = R(phid[l]);
      if constexpr (P::split)
        rho[l] = arho[l] / phi[l];
      else
        rho[l] = R(E(arho[l]) / phid[l]);
      ax.rho += arho[l];
    }
    bool ok = true;
#pragma unroll
    for (int h = 0; h < NH; ++h) {
      R ar = R(1);
#pragma unroll
      for (int l = 0; l < NMAT; ++l)
        if (a.hslot[l] == h) ar = arho[l];
      w[L::oH + 2 * h] = c[L::oH + 2 * h] / ar;
      w[L::oH + 2 * h + 1] = c[L::oH + 2 * h + 1] / ar;
    }
#pragma unroll
    for (int l = 0; l < NMAT; ++l) D[l] = damage_of(a, w, l);
#pragma unroll
    for (int k = 0; k < 3; ++k) ax.u[k] = k < DIM ? c[L::oMOM + k] / ax.rho : R(0);
    R X[9];
    fullX(c, X);
    Mix mx;
    if (!mixture(a, phi, rho, D, X, mx)) return false;
    E pE;
    if constexpr (P::split) {
      // rho e = rho E - rho |u|^2/2 with the one subtraction in FP64 (rho E
      // is kept in FP64 so its updates do not accumulate FP32 rounding)
      const R ke = R(0.5) * ax.rho * (ax.u[0] * ax.u[0] + ax.u[1] * ax.u[1] + ax.u[2] * ax.u[2]);
      R num = rhoE_d ? R(*rhoE_d - E(ke)) : R(cx[0]) - ke;
#pragma unroll
      for (int l = 0; l < NMAT; ++l)
        if (!isvoid(a, l)) num += -arho[l] * mx.e[l] + phi[l] * mx.gi[l] * mx.p[l];
      pE = E(num / mx.xi);
    } else {
      const E ke = 0.5 * E(ax.rho) *
                   (E(ax.u[0]) * E(ax.u[0]) + E(ax.u[1]) * E(ax.u[1]) + E(ax.u[2]) * E(ax.u[2]));
      E num = (rhoE_d ? *rhoE_d : E(cx[0])) - ke;
#pragma unroll
      for (int l = 0; l < NMAT; ++l)
        if (!isvoid(a, l)) num += -E(arho[l] * mx.e[l]) + E(phi[l]) * E(mx.p[l]) / E(mx.ga[l]);
      pE = num / E(mx.xi);
    }
#pragma unroll
    for (int l = 0; l < NPX; ++l) wx[1 + l] = phid[l];
#pragma unroll
    for (int l = 0; l < NMAT - 1; ++l) w[L::oPHI + l] = R(0);
#pragma unroll
    for (int l = 0; l < NMAT; ++l) w[L::oARHO + l] = rho[l];
#pragma unroll
    for (int k = 0; k < DIM; ++k) w[L::oMOM + k] = ax.u[k];
    w[L::oE] = R(0);
    wx[0] = XT(pE);
#pragma unroll
    for (int k = 0; k < L::NFC; ++k) w[L::oF + k] = c[L::oF + k];
#pragma unroll
    for (int k = 0; k < DIM; ++k) w[L::oX + k] = c[L::oX + k];
    // every value finite: a sum of them is finite exactly then (a NaN or an
    // infinity propagates; admissible states are far from overflowing it),
    // one test instead of one per value
    R sw = R(0);
#pragma unroll
    for (int k = 0; k < NF; ++k) sw += w[k] + c[k];
    XT sx = XT(0);
#pragma unroll
    for (int k = 0; k < NX; ++k) sx += cx[k] + wx[k];
    if (!(ok && mfinite(sw) && mfinite(sx))) return false;
    if (mxo) *mxo = mx;
    const R nu = VD && a.void_l >= 0 ? phi[VD ? a.void_l : 0] : R(0);
    return finish<AX>(a, R(pE), rho, arho, mx, ax, nu);
  }

  // Row AX of Fbar of a state vector.
  template <int AX>
  __device__ static __forceinline__ void frow(const R* c, R row[3]) {
#pragma unroll
    for (int j = 0; j < 3; ++j) {
      R v = R(0);
#pragma unroll
      for (int q = 0; q < L::NFC; ++q)
        if (FC<DIM>::idx(q) == 3 * AX + j) v = c[L::oF + q];
      row[j] = Fv(AX, j, v);
    }
  }

  // Physical flux along AX: q u_d for the advected densities, rho u_k u_d -
  // sigma_kd, rho E u_d - sigma_dj u_j, Fbar_ij u_d - Fbar_dj u_i (zero for
  // row d).
  template <int AX>
  __device__ static __forceinline__ void flux(const R* c, const XT* cx, const Aux<R>& ax, R* f,
                                              XT* fx) {
    const R ud = ax.u[AX];
#pragma unroll
    for (int l = 0; l < NPX; ++l) fx[1 + l] = cx[1 + l] * XT(ud);
#pragma unroll
    for (int l = 0; l < NMAT - 1; ++l) f[L::oPHI + l] = R(0);
#pragma unroll
    for (int l = 0; l < NMAT; ++l) f[L::oARHO + l] = c[L::oARHO + l] * ud;
#pragma unroll
    for (int k = 0; k < DIM; ++k) f[L::oMOM + k] = c[L::oMOM + k] * ud - ax.sd[k];
    f[L::oE] = R(0);
    if constexpr (P::split)
      fx[0] = XT(R(cx[0]) * ud - (ax.sr[0] * ax.u[0] + ax.sr[1] * ax.u[1] + ax.sr[2] * ax.u[2]));
    else
      fx[0] = cx[0] * E(ud) - (E(ax.sr[0]) * E(ax.u[0]) + E(ax.sr[1]) * E(ax.u[1]) +
                               E(ax.sr[2]) * E(ax.u[2]));
    R row[3];
    frow<AX>(c, row);
#pragma unroll
    for (int k = 0; k < L::NFC; ++k) {
      const int i = FC<DIM>::idx(k) / 3, j = FC<DIM>::idx(k) % 3;
      f[L::oF + k] = (i == AX) ? R(0) : Fv(i, j, c[L::oF + k]) * ud - row[j] * ax.u[i];
    }
#pragma unroll
    for (int k = 0; k < 2 * NH; ++k) f[L::oH + k] = c[L::oH + k] * ud;
#pragma unroll
    for (int k = 0; k < DIM; ++k) f[L::oX + k] = c[L::oX + k] * ud;
  }

  // Non-conservative terms per unit 1/dx: phi and X take q_c du; the
  // deformation tensor 2/3 Fbar_ij du - u_i dFbar_dj.
  template <int AX>
  __device__ static __forceinline__ void noncons(const R* wc, const XT* wcx, const R uc[3], R du,
                                                 const R dFrow[3], R* nc, XT* ncx) {
#pragma unroll
    for (int k = 0; k < NF; ++k) nc[k] = R(0);
    ncx[0] = XT(0);
#pragma unroll
    for (int l = 0; l < NPX; ++l) ncx[1 + l] = wcx[1 + l] * XT(du);
#pragma unroll
    for (int k = 0; k < DIM; ++k) nc[L::oX + k] = wc[L::oX + k] * du;
#pragma unroll
    for (int k = 0; k < L::NFC; ++k) {
      const int i = FC<DIM>::idx(k) / 3, j = FC<DIM>::idx(k) % 3;
      nc[L::oF + k] = (R(2) / R(3)) * Fv(i, j, wc[L::oF + k]) * du - uc[i] * dFrow[j];
    }
  }

  // Flux through the face from star side K (lft: the left star region
  // holds the face) of the subsonic fan: F_K + S_K (U*_K - U_K) plus the
  // jump across K's shear wave; the face velocity and the row d of Fbar of
  // that star region.
  template <int AX>
  __device__ static __forceinline__ void star_side(bool lft, const R* cL_, const XT* xL,
                                                   const Aux<R>& aL, const R* cR_, const XT* xR,
                                                   const Aux<R>& aR, R SL, R SR, R Ss, R* fo,
                                                   XT* fox, R& uface, R frowo[3]) {
    const R uL = aL.u[AX], uR = aR.u[AX];
    const R rL = aL.rho, rR = aR.rho;
    const R* cK = lft ? cL_ : cR_;
    const XT* xK = lft ? xL : xR;
    const Aux<R>& aK = lft ? aL : aR;
    flux<AX>(cK, xK, aK, fo, fox);
    frow<AX>(cK, frowo);
    const R uK = aK.u[AX];
    const R SK = lft ? SL : SR;
    const R chi = (SK - uK) / (SK - Ss);
    const R rK = aK.rho;
    // star state U*_K; the flux is F_K + S_K (U*_K - U_K)
    R us[NF];
#pragma unroll
    for (int l = 0; l < NMAT - 1; ++l) us[L::oPHI + l] = R(0);
#pragma unroll
    for (int l = 0; l < NPX; ++l) fox[1 + l] = fox[1 + l] + XT(SK) * (xK[1 + l] * XT(chi) - xK[1 + l]);
#pragma unroll
    for (int l = 0; l < NMAT; ++l) us[L::oARHO + l] = cK[L::oARHO + l] * chi;
#pragma unroll
    for (int k = 0; k < DIM; ++k) us[L::oMOM + k] = (k == AX) ? rK * chi * Ss : cK[L::oMOM + k] * chi;
    us[L::oE] = R(0);
    const XT Es = XT(chi) * (xK[0] + XT(rK) * XT(Ss) * (XT(Ss) - XT(uK)) -
                             XT(aK.sd[AX]) * (XT(Ss) - XT(uK)) / (XT(SK) - XT(uK)));
#pragma unroll
    for (int k = 0; k < L::NFC; ++k) {
      const int i = FC<DIM>::idx(k) / 3, j = FC<DIM>::idx(k) % 3;
      // Fbar* = Fbar chi off row d; in A form A* = (delta_ij + A_ij) chi - delta_ij
      if (i == AX)
        us[L::oF + k] = cK[L::oF + k];
      else
        us[L::oF + k] = AF ? Fv(i, j, cK[L::oF + k]) * chi - (i == j ? R(1) : R(0))
                           : cK[L::oF + k] * chi;
    }
#pragma unroll
    for (int k = 0; k < 2 * NH; ++k) us[L::oH + k] = cK[L::oH + k] * chi;
#pragma unroll
    for (int k = 0; k < DIM; ++k) us[L::oX + k] = cK[L::oX + k] * chi;
#pragma unroll
    for (int k = 0; k < NF; ++k)
      if (k != L::oE && (k < L::oPHI || k >= L::oPHI + L::NPHI)) fo[k] = fo[k] + SK * (us[k] - cK[k]);
    fox[0] = fox[0] + XT(SK) * (Es - xK[0]);
    uface = uK + SK * (chi - R(1));
    if (DIM == 1) return;
    // shear waves in the star regions
    const R rsL = rL * ((SL - uL) / (SL - Ss));
    const R rsR = rR * ((SR - uR) / (SR - Ss));
    R csL = msqrt(aL.G / rsL), csR = msqrt(aR.G / rsR);
    if (csL > Ss - SL) csL = Ss - SL;
    if (csR > SR - Ss) csR = SR - Ss;
    const R ZL = rsL * csL, ZR = rsR * csR;
    if (!(ZL + ZR > R(0))) return;
    if (lft ? !(Ss - csL < R(0)) : !(Ss + csR > R(0))) return;
    const R csK = lft ? csL : csR;
    // a side without shear stiffness has no shear wave (it would coincide
    // with the contact; reached at a contact at rest)
    if (!(csK > R(0))) return;
    const R rsK = lft ? rsL : rsR;
    const R sgn = lft ? R(1) : R(-1);
    const R SSK = lft ? Ss - csL : Ss + csR;
    XT ess = Es;
#pragma unroll
    for (int t = 0; t < DIM; ++t) {
      if (t == AX) continue;
      const R uLt = aL.u[t], uRt = aR.u[t];
      const R tauL = aL.sd[t], tauR = aR.sd[t];
      const R uss = (tauR - tauL + ZL * uLt + ZR * uRt) / (ZL + ZR);
      const R tss = tauL + ZL * (uss - uLt);
      const R uKt = lft ? uLt : uRt, tauK = lft ? tauL : tauR;
      const R du = uss - uKt;
      fo[L::oMOM + t] = fo[L::oMOM + t] + SSK * (rsK * uss - us[L::oMOM + t]);
#pragma unroll
      for (int k = 0; k < L::NFC; ++k) {
        const int i = FC<DIM>::idx(k) / 3, j = FC<DIM>::idx(k) % 3;
        if (i == t) {
          const R uss_f = us[L::oF + k] + sgn * frowo[j] * du / csK;
          fo[L::oF + k] = fo[L::oF + k] + SSK * (uss_f - us[L::oF + k]);
        }
      }
      ess += XT(sgn) * (XT(tss) * XT(uss) - XT(tauK) * XT(uKt)) / XT(csK);
    }
    fox[0] = fox[0] + XT(SSK) * (ess - Es);
  }

  // ---- void opening (void grids): Sec. 3.1 opens void where either face
  // state is critically damaged and the two are in tension along the sweep,
  // x^T (sigma_L + sigma_R) x > 0.  Each side meets a traction-free surface;
  // where the surfaces separate the gap between them is void.

  // A damaged solid at D >= D_cut = D_crit (1 - 1e-4), as in the yield
  // stress.
  __device__ static __forceinline__ bool critical(const KArgs& a, const R* c) {
    bool crit = false;
#pragma unroll
    for (int l = 0; l < NMAT; ++l) {
      const auto& m = matp<R>(a, l);
#pragma unroll
      for (int h = 0; h < NH; ++h)
        if (a.hslot[l] == h && m.damage != 0) {
          const R ar = c[L::oARHO + l];
          if (ar > R(0)) crit = crit || c[L::oH + 2 * h + 1] / ar >= R(m.D_cut);
        }
    }
    return crit;
  }

  // Speed of side K's traction-free surface: across K's longitudinal wave
  // S_K = u_K -/+ c_L,K the normal stress drops to zero (HLLC jump relation
  // 0 = sigma_K - rho_K (S_K - u_K)(S_f - u_K)).
  template <int AX>
  __device__ static __forceinline__ R free_surface_speed(bool lft, const Aux<R>& ax) {
    const R SK = lft ? ax.u[AX] - ax.cL : ax.u[AX] + ax.cL;
    return ax.u[AX] + ax.sd[AX] / (ax.rho * (SK - ax.u[AX]));
  }

  // Flux of side K's fan against a traction-free surface: waves S_K, the
  // shear wave S_f -/+ c_s and the surface S_f; the normal stress and then
  // the tangential tractions are zero behind them.  at_face: the region
  // holding x/t = 0; otherwise the region just inside the surface.
  template <int AX>
  __device__ static void free_surface_flux(bool lft, const R* cK, const XT* xK, const Aux<R>& aK,
                                           bool at_face, R* fo, XT* fox, R& uface,
                                           R frowo[3]) {
    const R uK = aK.u[AX];
    const R SK = lft ? uK - aK.cL : uK + aK.cL;
    const R Sf = free_surface_speed<AX>(lft, aK);
    flux<AX>(cK, xK, aK, fo, fox);
    frow<AX>(cK, frowo);
    uface = uK;
    if (at_face && (lft ? SK >= R(0) : SK <= R(0))) return;  // region K
    const R chi = (SK - uK) / (SK - Sf);
    const R rK = aK.rho;
    R us[NF];
#pragma unroll
    for (int l = 0; l < NMAT - 1; ++l) us[L::oPHI + l] = R(0);
#pragma unroll
    for (int l = 0; l < NPX; ++l) fox[1 + l] = fox[1 + l] + XT(SK) * (xK[1 + l] * XT(chi) - xK[1 + l]);
#pragma unroll
    for (int l = 0; l < NMAT; ++l) us[L::oARHO + l] = cK[L::oARHO + l] * chi;
#pragma unroll
    for (int k = 0; k < DIM; ++k) us[L::oMOM + k] = (k == AX) ? rK * chi * Sf : cK[L::oMOM + k] * chi;
    us[L::oE] = R(0);
    const XT Es = XT(chi) * (xK[0] + XT(rK) * XT(Sf) * (XT(Sf) - XT(uK)) -
                             XT(aK.sd[AX]) * (XT(Sf) - XT(uK)) / (XT(SK) - XT(uK)));
#pragma unroll
    for (int k = 0; k < L::NFC; ++k) {
      const int i = FC<DIM>::idx(k) / 3, j = FC<DIM>::idx(k) % 3;
      if (i == AX)
        us[L::oF + k] = cK[L::oF + k];
      else
        us[L::oF + k] = AF ? Fv(i, j, cK[L::oF + k]) * chi - (i == j ? R(1) : R(0))
                           : cK[L::oF + k] * chi;
    }
#pragma unroll
    for (int k = 0; k < 2 * NH; ++k) us[L::oH + k] = cK[L::oH + k] * chi;
#pragma unroll
    for (int k = 0; k < DIM; ++k) us[L::oX + k] = cK[L::oX + k] * chi;
#pragma unroll
    for (int k = 0; k < NF; ++k)
      if (k != L::oE && (k < L::oPHI || k >= L::oPHI + L::NPHI)) fo[k] = fo[k] + SK * (us[k] - cK[k]);
    fox[0] = fox[0] + XT(SK) * (Es - xK[0]);
    uface = uK + SK * (chi - R(1));
    if (DIM == 1) return;
    // the shear wave: speed from the star density, kept between S_K and S_f
    const R rs = rK * ((SK - uK) / (SK - Sf));
    R cs = msqrt(aK.G / rs);
    if (cs > mabs(Sf - SK)) cs = mabs(Sf - SK);
    if (!(cs > R(0))) return;
    const R SSK = lft ? Sf - cs : Sf + cs;
    if (at_face && (lft ? SSK >= R(0) : SSK <= R(0))) return;  // region K*
    const R Z = rs * cs, sgn = lft ? R(1) : R(-1);
    XT ess = Es;
#pragma unroll
    for (int t = 0; t < DIM; ++t) {
      if (t == AX) continue;
      const R tau = aK.sd[t], ut = aK.u[t];
      // zero traction behind the shear wave: tau + sgn Z (uss - ut) = 0
      const R uss = ut - sgn * tau / Z;
      const R du = uss - ut;
      fo[L::oMOM + t] = fo[L::oMOM + t] + SSK * (rs * uss - us[L::oMOM + t]);
#pragma unroll
      for (int k = 0; k < L::NFC; ++k) {
        const int i = FC<DIM>::idx(k) / 3, j = FC<DIM>::idx(k) % 3;
        if (i == t) {
          const R uss_f = us[L::oF + k] + sgn * frowo[j] * du / cs;
          fo[L::oF + k] = fo[L::oF + k] + SSK * (uss_f - us[L::oF + k]);
        }
      }
      ess += XT(sgn) * (XT(0) * XT(uss) - XT(tau) * XT(ut)) / XT(cs);
    }
    fox[0] = fox[0] + XT(SSK) * (ess - Es);
  }

  // The face's two records, as the cell left of it sees it (fL, fxL, ufL,
  // rowL) and as the cell right of it does.  Both are the contact solver's
  // unless the void opens.  Where it opens, each side's surface sets that
  // side's face velocity, Fbar and X transport; the conserved fields and
  // the material fractions take what crosses the face (nothing when the gap
  // holds it, else the fan of the side whose surface has passed it), and
  // the void fraction takes the rest: a side receiving the gap gets void at
  // the rate S_f,own - u_crossing, so its fractions keep summing to one.
  template <int AX>
  __device__ static void riemann2(const KArgs& a, const R* cL_, const XT* xL, const Aux<R>& aL,
                                  const R* cR_, const XT* xR, const Aux<R>& aR, R* fL, XT* fxL,
                                  R& ufL, R rowL[3], R* fR, XT* fxR, R& ufR, R rowR[3]) {
    if (a.void_l >= 0 && (critical(a, cL_) || critical(a, cR_)) && aL.sd[AX] + aR.sd[AX] > R(0)) {
      const R SfL = free_surface_speed<AX>(true, aL), SfR = free_surface_speed<AX>(false, aR);
      if (SfL < SfR) {
        // the crossing side's fan at the face (nothing if the gap holds it)
        R fc[NF], ufc = R(0), rowc[3];
        XT fxc[NX];
        int cross = -1;
#pragma unroll
        for (int k = 0; k < NF; ++k) fc[k] = R(0);
#pragma unroll
        for (int k = 0; k < NX; ++k) fxc[k] = XT(0);
        if (SfL > R(0)) {
          cross = 0;
          free_surface_flux<AX>(true, cL_, xL, aL, true, fc, fxc, ufc, rowc);
        } else if (SfR < R(0)) {
          cross = 1;
          free_surface_flux<AX>(false, cR_, xR, aR, true, fc, fxc, ufc, rowc);
        }
#pragma unroll 1
        for (int side = 0; side < 2; ++side) {
          const bool lft = side == 0;
          R* fo = lft ? fL : fR;
          XT* fox = lft ? fxL : fxR;
          R& uf = lft ? ufL : ufR;
          R* row = lft ? rowL : rowR;
          R fs[NF], ufs, rows[3];
          XT fxs[NX];
          free_surface_flux<AX>(lft, lft ? cL_ : cR_, lft ? xL : xR, lft ? aL : aR, false, fs, fxs,
                                ufs, rows);
#pragma unroll
          for (int j = 0; j < 3; ++j) row[j] = rows[j];
          if (cross == side) {
#pragma unroll
            for (int k = 0; k < NF; ++k) fo[k] = fc[k];
#pragma unroll
            for (int k = 0; k < NX; ++k) fox[k] = fxc[k];
            uf = ufc;
            continue;
          }
#pragma unroll
          for (int k = 0; k < NF; ++k)
            fo[k] = ((k >= L::oF && k < L::oF + L::NFC) || k >= L::oX) ? fs[k] : fc[k];
#pragma unroll
          for (int k = 0; k < NX; ++k) fox[k] = fxc[k];
#pragma unroll
          for (int l = 0; l < NPX; ++l)
            if (l == a.void_l) fox[1 + l] = fox[1 + l] + XT(ufs - ufc);
          uf = ufs;
        }
        return;
      }
    }
    riemann<AX>(cL_, xL, aL, cR_, xR, aR, fL, fxL, ufL, rowL);
#pragma unroll
    for (int k = 0; k < NF; ++k) fR[k] = fL[k];
#pragma unroll
    for (int k = 0; k < NX; ++k) fxR[k] = fxL[k];
    ufR = ufL;
#pragma unroll
    for (int j = 0; j < 3; ++j) rowR[j] = rowL[j];
  }

  // HLLD-type Riemann solver for the elastic mixture: outer waves S_L, S_R
  // (Davis), contact S*, shear waves S* -/+ c_s inside the star regions.
  // Jumps from the Rankine-Hugoniot conditions of each wave; with G = 0 it
  // is the HLLC solver.  Outputs the flux, the normal velocity at the face
  // and the row d of Fbar of the star region holding the face.  A contact
  // at rest (S* zero to within the rounding of the wave speeds: a reflective
  // wall, a symmetry plane, still gas) lies on the face itself, which then
  // takes the mean of what the two star sides give: it does not depend on
  // the sign of a rounded zero, and at a wall the tangential rows of Fbar
  // have no flux.
  template <int AX>
  __device__ static void riemann(const R* cL_, const XT* xL, const Aux<R>& aL, const R* cR_,
                                 const XT* xR, const Aux<R>& aR, R* fo, XT* fox, R& uface,
                                 R frowo[3]) {
    const R uL = aL.u[AX], uR = aR.u[AX];
    const R a1 = uL - aL.cL, a2 = uR - aR.cL;
    const R b1 = uL + aL.cL, b2 = uR + aR.cL;
    const R SL = a1 < a2 ? a1 : a2;
    const R SR = b1 > b2 ? b1 : b2;
    const R sL = aL.sd[AX], sR = aR.sd[AX];
    const R rL = aL.rho, rR = aR.rho;
    R Ss;
    if constexpr (P::split) {
      // separately rounded products (no contraction): the numerator is then
      // exactly odd under the mirror of the face, and exactly zero where the
      // two sides are mirror images (a wall, a symmetry plane) in every
      // kernel, whatever the compiler fuses elsewhere
      const float X = __fmul_rn(__fmul_rn(rL, uL), __fsub_rn(SL, uL));
      const float Y = __fmul_rn(__fmul_rn(rR, uR), __fsub_rn(SR, uR));
      const float num = __fadd_rn(__fsub_rn(sL, sR), __fsub_rn(X, Y));
      const float den = __fsub_rn(__fmul_rn(rL, __fsub_rn(SL, uL)), __fmul_rn(rR, __fsub_rn(SR, uR)));
      Ss = num / den;
    } else {
      Ss = (sL - sR + rL * uL * (SL - uL) - rR * uR * (SR - uR)) /
           (rL * (SL - uL) - rR * (SR - uR));
    }
    if (SL >= R(0) || SR <= R(0)) {
      // supersonic: the state on the upwind side of both waves
      const bool lft = SL >= R(0);
      const Aux<R>& aK = lft ? aL : aR;
      flux<AX>(lft ? cL_ : cR_, lft ? xL : xR, aK, fo, fox);
      frow<AX>(lft ? cL_ : cR_, frowo);
      uface = aK.u[AX];
      return;
    }
    // at rest: |S*| <= 16 eps (S_R - S_L) with eps = 2^-52 in both
    // precisions (the FP32 path takes it as the exact zero of a wall or a
    // symmetry plane; an FP32-rounding threshold would average the sides
    // of slowly moving contacts)
    const bool rest = mabs(Ss) <= R(16.0 * Eps<double>::unit) * (SR - SL);
    // one star side, or both (weights 1/2 each, exact) for a contact at rest;
    // one code copy for either
#pragma unroll 1
    for (int side = 0; side < (rest ? 2 : 1); ++side) {
      const bool lft = rest ? side == 0 : Ss >= R(0);
      R f[NF], row[3], uf;
      XT fx[NX];
      star_side<AX>(lft, cL_, xL, aL, cR_, xR, aR, SL, SR, Ss, f, fx, uf, row);
      const R wg = rest ? R(0.5) : R(1);
      const XT wgx = rest ? XT(0.5) : XT(1);
#pragma unroll
      for (int k = 0; k < NF; ++k) fo[k] = (side == 0 ? R(0) : fo[k]) + wg * f[k];
#pragma unroll
      for (int k = 0; k < NX; ++k) fox[k] = (side == 0 ? XT(0) : fox[k]) + wgx * fx[k];
#pragma unroll
      for (int j = 0; j < 3; ++j) frowo[j] = (side == 0 ? R(0) : frowo[j]) + wg * row[j];
      uface = (side == 0 ? R(0) : uface) + wg * uf;
    }
  }
};

}  // namespace mm
