// mpm_math.cuh -- FP32 device math of the MLS-MPM substep and its adjoint.
//
// arXiv 2412.12089, App. D.3: MLS-MPM transfers (quadratic B-splines, APIC affine
// momentum), the von Mises elastoplastic law (Hencky stress + return mapping), the
// weakly compressible fluid (P = lam J (J - 1) F^-T, projection J^(1/3) I), a
// compressible neo-Hookean solid and a neo-Hookean muscle with active fibre stress, and
// the softened contact s = min(exp(-alpha d), 1).  The reverse-mode helpers are the
// exact derivatives of these FP32 functions (Sec. 4.1, discrete adjoint).
#pragma once
#include <cuda_runtime.h>
#include <math.h>

namespace mpm {

#define MPM_HD __device__ __forceinline__

// ------------------------------------------------------------------ 3x3 helpers
// Matrices are float[9], row-major: M[3*i + j] = M_ij.

MPM_HD float det3(const float* A) {
  return A[0] * (A[4] * A[8] - A[5] * A[7]) - A[1] * (A[3] * A[8] - A[5] * A[6]) +
         A[2] * (A[3] * A[7] - A[4] * A[6]);
}

// Cofactor matrix cof(A) = det(A) A^{-T}.
MPM_HD void cofactor3(const float* A, float* K) {
  K[0] = A[4] * A[8] - A[5] * A[7];
  K[1] = A[5] * A[6] - A[3] * A[8];
  K[2] = A[3] * A[7] - A[4] * A[6];
  K[3] = A[2] * A[7] - A[1] * A[8];
  K[4] = A[0] * A[8] - A[2] * A[6];
  K[5] = A[1] * A[6] - A[0] * A[7];
  K[6] = A[1] * A[5] - A[2] * A[4];
  K[7] = A[2] * A[3] - A[0] * A[5];
  K[8] = A[0] * A[4] - A[1] * A[3];
}

MPM_HD void matmul3(const float* A, const float* B, float* O) {
#pragma unroll
  for (int i = 0; i < 3; ++i)
#pragma unroll
    for (int j = 0; j < 3; ++j)
      O[3 * i + j] = A[3 * i] * B[j] + A[3 * i + 1] * B[3 + j] + A[3 * i + 2] * B[6 + j];
}

// ------------------------------------------------------------------ quadratic B-spline

// Weights of nodes base+0..2 at fx = X - base in [0.5, 1.5) and their d/dfx.
MPM_HD void bspline(float fx, float* w, float* dw) {
  float a = 1.5f - fx, b = fx - 1.0f, c = fx - 0.5f;
  w[0] = 0.5f * a * a;
  w[1] = 0.75f - b * b;
  w[2] = 0.5f * c * c;
  dw[0] = -a;
  dw[1] = -2.0f * b;
  dw[2] = c;
}

// Cell base along one axis: floor(x*G - 0.5) with each operation rounded separately
// (the binning depends on it bit for bit), clamped into [0, G-3].  *oob is set on clamp.
MPM_HD int cell_base(float x, float G, int Gi, int* oob) {
  float X = __fmul_rn(x, G);
  float fb = floorf(__fsub_rn(X, 0.5f));
  int b;
  if (!(fb >= 0.0f)) {  // negative or NaN
    b = 0;
    *oob = 1;
  } else if (fb > (float)(Gi - 3)) {
    b = Gi - 3;
    *oob = 1;
  } else {
    b = (int)fb;
  }
  return b;
}

// ------------------------------------------------------------------ deformation in H = F - I
// The deformation gradient is stored and processed as its displacement part H = F - I.
// Near the undeformed state (the common case) FP32 holds H to ~1e-7 of |H|, while F itself
// would carry an absolute error of one ulp of 1 (6e-8): on the light materials of the
// paper's tasks (rho = 1) that much strain error is already a visible stress.  Every law
// below is written so that small deformations are never formed as 1 + small - 1.

// det(I + H) - 1 = tr H + (sum of principal 2x2 minors) + det H
MPM_HD float detm1(const float* H) {
  const float tr = H[0] + H[4] + H[8];
  const float m2 = H[0] * H[4] - H[1] * H[3] + H[0] * H[8] - H[2] * H[6] + H[4] * H[8] - H[5] * H[7];
  return tr + m2 + det3(H);
}

// F = I + H
MPM_HD void f_of(const float* H, float* F) {
#pragma unroll
  for (int i = 0; i < 9; ++i) F[i] = H[i] + ((i % 4 == 0) ? 1.0f : 0.0f);
}

// B = H + H^T + H H^T = F F^T - I (symmetric; stored full)
MPM_HD void left_strain(const float* H, float* B) {
#pragma unroll
  for (int i = 0; i < 3; ++i)
#pragma unroll
    for (int j = 0; j < 3; ++j)
      B[3 * i + j] = H[3 * i + j] + H[3 * j + i] + H[3 * i] * H[3 * j] + H[3 * i + 1] * H[3 * j + 1] +
                     H[3 * i + 2] * H[3 * j + 2];
}

// Symmetric 3x3 eigen-decomposition by cyclic Jacobi rotations: A = U diag(lam) U^T,
// eigenvectors in the columns of U.  A is destroyed.
template <int P, int Q>
MPM_HD void sym_rot(float* A, float* U) {
  const float apq = A[3 * P + Q];
  if (apq == 0.0f) return;
  const float app = A[3 * P + P], aqq = A[3 * Q + Q];
  const float th = (aqq - app) / (2.0f * apq);
  const float t = fabsf(th) > 1e10f ? 0.5f / th : copysignf(1.0f, th) / (fabsf(th) + sqrtf(th * th + 1.0f));
  const float c = rsqrtf(t * t + 1.0f), s = t * c;
  constexpr int R = 3 - P - Q;
  A[3 * P + P] = app - t * apq;
  A[3 * Q + Q] = aqq + t * apq;
  A[3 * P + Q] = A[3 * Q + P] = 0.0f;
  const float arp = A[3 * R + P], arq = A[3 * R + Q];
  A[3 * R + P] = A[3 * P + R] = c * arp - s * arq;
  A[3 * R + Q] = A[3 * Q + R] = s * arp + c * arq;
#pragma unroll
  for (int k = 0; k < 3; ++k) {
    const float up = U[3 * k + P], uq = U[3 * k + Q];
    U[3 * k + P] = c * up - s * uq;
    U[3 * k + Q] = s * up + c * uq;
  }
}

MPM_HD void sym_eig3(float* A, float* lam, float* U) {
#pragma unroll
  for (int i = 0; i < 9; ++i) U[i] = (i % 4 == 0) ? 1.0f : 0.0f;
#pragma unroll 1
  for (int sweep = 0; sweep < 8; ++sweep) {
    const float off = fabsf(A[1]) + fabsf(A[2]) + fabsf(A[5]);
    const float dia = fabsf(A[0]) + fabsf(A[4]) + fabsf(A[8]);
    if (!(off > 1e-9f * dia) || !(off > 1e-37f)) break;
    sym_rot<0, 1>(A, U);
    sym_rot<0, 2>(A, U);
    sym_rot<1, 2>(A, U);
  }
  lam[0] = A[0];
  lam[1] = A[4];
  lam[2] = A[8];
}

// U diag(d) W^T
MPM_HD void udvt(const float* U, const float* d, const float* W, float* O) {
#pragma unroll
  for (int i = 0; i < 3; ++i)
#pragma unroll
    for (int j = 0; j < 3; ++j)
      O[3 * i + j] = U[3 * i] * d[0] * W[3 * j] + U[3 * i + 1] * d[1] * W[3 * j + 1] + U[3 * i + 2] * d[2] * W[3 * j + 2];
}

// M = U^T A W
MPM_HD void ut_a_w(const float* U, const float* A, const float* W, float* M) {
  float T[9];
#pragma unroll
  for (int i = 0; i < 3; ++i)
#pragma unroll
    for (int j = 0; j < 3; ++j)
      T[3 * i + j] = U[i] * A[j] + U[3 + i] * A[3 + j] + U[6 + i] * A[6 + j];  // (U^T A)_ij
#pragma unroll
  for (int i = 0; i < 3; ++i)
#pragma unroll
    for (int j = 0; j < 3; ++j)
      M[3 * i + j] = T[3 * i] * W[j] + T[3 * i + 1] * W[3 + j] + T[3 * i + 2] * W[6 + j];
}

// log((1+a)/(1+b))/(a - b) without cancellation (-> 1/(1+b) as a -> b).
MPM_HD float log1p_ratio(float a, float b) {
  const float d = a - b;
  const float z = d / (1.0f + b);
  if (fabsf(z) < 1e-3f) return (1.0f - z * (0.5f - z * (1.0f / 3.0f))) / (1.0f + b);
  return log1pf(z) / d;
}

// expm1(z)/z without cancellation.
MPM_HD float expm1_ratio(float z) {
  if (fabsf(z) < 1e-3f) return 1.0f + z * (0.5f + z * (1.0f / 6.0f));
  return expm1f(z) / z;
}

// Polar data of F = I + H: F = U diag(s) V^T with U, beta from B = F F^T - I = U diag(beta) U^T,
// s = sqrt(1 + beta) and Hencky strains eps = log s = log1p(beta)/2 (s clamped at kSigMin).
constexpr float kSigMin = 1e-4f;
constexpr float kBetaMin = kSigMin * kSigMin - 1.0f;

struct Polar {
  float U[9];
  float beta[3], s[3], eps[3];
};

MPM_HD void polar(const float* H, Polar& P) {
  float B[9];
  left_strain(H, B);
  sym_eig3(B, P.beta, P.U);
#pragma unroll
  for (int i = 0; i < 3; ++i) {
    const float b = fmaxf(P.beta[i], kBetaMin);
    P.beta[i] = b;
    P.s[i] = sqrtf(1.0f + b);
    P.eps[i] = 0.5f * log1pf(b);
  }
}

// ------------------------------------------------------------------ materials

enum { MAT_NEOHOOKEAN = 0, MAT_VONMISES = 1, MAT_FLUID = 2, MAT_MUSCLE = 3 };

struct Mat {
  int kind;
  float mu, lam;
  float cyl;  // von Mises threshold c_y * sigma_y / (2 mu) on |eps^|
  float bulk, visc, act;
};

// Kirchhoff stress tau(F = I + H, C) of the material (laws in mpm.h).
MPM_HD void kirchhoff(const Mat& m, const float* H, const float* C, float a_g, float* tau) {
  if (m.kind == MAT_VONMISES) {
    Polar P;
    polar(H, P);
    const float tr = m.lam * (P.eps[0] + P.eps[1] + P.eps[2]);
    const float t[3] = {2.0f * m.mu * P.eps[0] + tr, 2.0f * m.mu * P.eps[1] + tr, 2.0f * m.mu * P.eps[2] + tr};
    udvt(P.U, t, P.U, tau);
  } else if (m.kind == MAT_FLUID) {
    const float Jm1 = detm1(H);
    const float J = 1.0f + Jm1;
    const float p = m.bulk * J * Jm1;
    const float vj = m.visc * J;
#pragma unroll
    for (int i = 0; i < 3; ++i)
#pragma unroll
      for (int j = 0; j < 3; ++j) tau[3 * i + j] = (i == j ? p : 0.0f) + vj * (C[3 * i + j] + C[3 * j + i]);
  } else {  // neo-Hookean: mu (F F^T - I) + lam log J I, F F^T - I = H + H^T + H H^T (+ muscle fibre)
    float B[9];
    left_strain(H, B);
    const float lj = m.lam * log1pf(detm1(H));
#pragma unroll
    for (int i = 0; i < 9; ++i) tau[i] = m.mu * B[i] + ((i % 4 == 0) ? lj : 0.0f);
    if (m.kind == MAT_MUSCLE && a_g != 0.0f) {
      const float k = a_g * m.act;
      const float f[3] = {H[2], H[5], 1.0f + H[8]};  // F e_z
#pragma unroll
      for (int i = 0; i < 3; ++i)
#pragma unroll
        for (int j = 0; j < 3; ++j) tau[3 * i + j] += k * f[i] * f[j];
    }
  }
}

// Adjoint of kirchhoff(): Hb += dtau/dH^T tb (= dtau/dF^T tb), Cb += dtau/dC^T tb,
// *agb += dtau/da_g . tb.
MPM_HD void kirchhoff_vjp(const Mat& m, const float* H, const float* C, float a_g, const float* tb, float* Hb,
                          float* Cb, float* agb) {
  if (m.kind == MAT_VONMISES) {
    // tau = U diag(t) U^T, F = U diag(s) V^T, V^T = diag(1/s) U^T F.  Rotated frame:
    // M = U^T tb U; K_kk = sum_i M_ii dt_i/ds_k; pair (i,j): with
    // Q = (t_j - t_i)/(s_j^2 - s_i^2) = mu log((1+b_j)/(1+b_i))/(b_j - b_i),
    // K_ij = Q s_j (M_ij + M_ji), K_ji = Q s_i (M_ij + M_ji).  Fb = U K V^T.
    Polar P;
    polar(H, P);
    float M[9];
    ut_a_w(P.U, tb, P.U, M);
    float K[9];
    const float trM = M[0] + M[4] + M[8];
#pragma unroll
    for (int k = 0; k < 3; ++k) {
      const float de = P.beta[k] > kBetaMin ? 1.0f / P.s[k] : 0.0f;  // d eps_k / d s_k
      K[4 * k] = (2.0f * m.mu * M[4 * k] + m.lam * trM) * de;
    }
    const int PI[3] = {0, 0, 1}, PJ[3] = {1, 2, 2};
#pragma unroll
    for (int r = 0; r < 3; ++r) {
      const int i = PI[r], j = PJ[r];
      const float Q = m.mu * log1p_ratio(P.beta[j], P.beta[i]);
      const float sym = M[3 * i + j] + M[3 * j + i];
      K[3 * i + j] = Q * P.s[j] * sym;
      K[3 * j + i] = Q * P.s[i] * sym;
    }
    // Fb = U K diag(1/s) U^T F
    float F[9], W[9], T[9], R[9];
    f_of(H, F);
#pragma unroll
    for (int a = 0; a < 3; ++a)
#pragma unroll
      for (int b = 0; b < 3; ++b) W[3 * a + b] = K[3 * a + b] / P.s[b];
    matmul3(P.U, W, T);
#pragma unroll
    for (int a = 0; a < 3; ++a)
#pragma unroll
      for (int b = 0; b < 3; ++b) R[3 * a + b] = T[3 * a] * P.U[3 * b] + T[3 * a + 1] * P.U[3 * b + 1] + T[3 * a + 2] * P.U[3 * b + 2];
    matmul3(R, F, T);
#pragma unroll
    for (int i = 0; i < 9; ++i) Hb[i] += T[i];
  } else if (m.kind == MAT_FLUID) {
    const float Jm1 = detm1(H);
    const float J = 1.0f + Jm1;
    const float tr = tb[0] + tb[4] + tb[8];
    float cc = 0.0f;
#pragma unroll
    for (int i = 0; i < 3; ++i)
#pragma unroll
      for (int j = 0; j < 3; ++j) cc += tb[3 * i + j] * (C[3 * i + j] + C[3 * j + i]);
    const float Jb = m.bulk * (2.0f * J - 1.0f) * tr + m.visc * cc;
    float F[9], K[9];
    f_of(H, F);
    cofactor3(F, K);  // dJ/dF
#pragma unroll
    for (int i = 0; i < 9; ++i) Hb[i] += Jb * K[i];
    const float vj = m.visc * J;
#pragma unroll
    for (int i = 0; i < 3; ++i)
#pragma unroll
      for (int j = 0; j < 3; ++j) Cb[3 * i + j] += vj * (tb[3 * i + j] + tb[3 * j + i]);
  } else {
    // tau = mu (F F^T - I) + lam log J I  ->  Fb += mu (tb + tb^T) F + lam tr(tb) cof(F) / J
    float S[9], F[9], K[9];
#pragma unroll
    for (int i = 0; i < 3; ++i)
#pragma unroll
      for (int j = 0; j < 3; ++j) S[3 * i + j] = tb[3 * i + j] + tb[3 * j + i];
    f_of(H, F);
    cofactor3(F, K);
    const float c = m.lam * (tb[0] + tb[4] + tb[8]) / (1.0f + detm1(H));
#pragma unroll
    for (int i = 0; i < 3; ++i)
#pragma unroll
      for (int j = 0; j < 3; ++j)
        Hb[3 * i + j] += m.mu * (S[3 * i] * F[j] + S[3 * i + 1] * F[3 + j] + S[3 * i + 2] * F[6 + j]) + c * K[3 * i + j];
    if (m.kind == MAT_MUSCLE) {
      const float f[3] = {F[2], F[5], F[8]};
      float Sf[3];
#pragma unroll
      for (int i = 0; i < 3; ++i) Sf[i] = S[3 * i] * f[0] + S[3 * i + 1] * f[1] + S[3 * i + 2] * f[2];
      const float k = a_g * m.act;
      Hb[2] += k * Sf[0];
      Hb[5] += k * Sf[1];
      Hb[8] += k * Sf[2];
      *agb += 0.5f * m.act * (f[0] * Sf[0] + f[1] * Sf[1] + f[2] * Sf[2]);  // f^T tb f
    }
  }
}

// Plastic projection of the trial H (after the F update in G2P), H -> H_out.
//  VONMISES: when |eps^| > cyl, F_out = U exp(eps_new) V^T = (I + D) F with
//            D = U diag(expm1(eps_new - eps)) U^T and eps_new - eps = (cyl/|eps^| - 1) eps^,
//            so H_out = D + H + D H.
//  FLUID:    F_out = J^(1/3) I, H_out = expm1(log1p(J - 1)/3) I.
MPM_HD void project(const Mat& m, const float* Ht, float* Ho) {
  if (m.kind == MAT_VONMISES) {
    Polar P;
    polar(Ht, P);
    const float mean = (P.eps[0] + P.eps[1] + P.eps[2]) * (1.0f / 3.0f);
    const float h0 = P.eps[0] - mean, h1 = P.eps[1] - mean, h2 = P.eps[2] - mean;
    const float nh = sqrtf(h0 * h0 + h1 * h1 + h2 * h2);
    if (!(nh > m.cyl)) {
#pragma unroll
      for (int i = 0; i < 9; ++i) Ho[i] = Ht[i];
      return;
    }
    const float km1 = m.cyl / nh - 1.0f;
    const float dg[3] = {expm1f(km1 * h0), expm1f(km1 * h1), expm1f(km1 * h2)};
    float D[9], DH[9];
    udvt(P.U, dg, P.U, D);
    matmul3(D, Ht, DH);
#pragma unroll
    for (int i = 0; i < 9; ++i) Ho[i] = D[i] + Ht[i] + DH[i];
  } else if (m.kind == MAT_FLUID) {
    const float c = expm1f(log1pf(detm1(Ht)) * (1.0f / 3.0f));
#pragma unroll
    for (int i = 0; i < 9; ++i) Ho[i] = (i % 4 == 0) ? c : 0.0f;
  } else {
#pragma unroll
    for (int i = 0; i < 9; ++i) Ho[i] = Ht[i];
  }
}

// Htb = dProject/dH^T Hob.
MPM_HD void project_vjp(const Mat& m, const float* Ht, const float* Hob, float* Htb) {
  if (m.kind == MAT_VONMISES) {
    Polar P;
    polar(Ht, P);
    const float mean = (P.eps[0] + P.eps[1] + P.eps[2]) * (1.0f / 3.0f);
    const float h[3] = {P.eps[0] - mean, P.eps[1] - mean, P.eps[2] - mean};
    const float nh = sqrtf(h[0] * h[0] + h[1] * h[1] + h[2] * h[2]);
    if (!(nh > m.cyl)) {
#pragma unroll
      for (int i = 0; i < 9; ++i) Htb[i] = Hob[i];
      return;
    }
    // G(F) = U diag(g) V^T, g_i = exp(mean + k eps^_i), k = cyl/|eps^|.
    //  dg_i/ds_k = g_i (1/3 + cyl (delta_ik - n_i n_k - 1/3)/|eps^|) / s_k
    //  A_ij = (g_i - g_j)/(s_i - s_j) = g_j k R_ij expm1(z)/z, z = k (eps_i - eps_j),
    //         R_ij = (eps_i - eps_j)/(s_i - s_j) = (s_i + s_j)/2 log((1+b_i)/(1+b_j))/(b_i - b_j)
    //  B_ij = (g_i + g_j)/(s_i + s_j)
    // with V^T = diag(1/s) U^T F:  M = U^T Gb V,  Fb = U K V^T.
    const float k = m.cyl / nh;
    const float n[3] = {h[0] / nh, h[1] / nh, h[2] / nh};
    const float g[3] = {P.s[0] * expf((k - 1.0f) * h[0]), P.s[1] * expf((k - 1.0f) * h[1]), P.s[2] * expf((k - 1.0f) * h[2])};
    float F[9], T[9], M[9];
    f_of(Ht, F);
    // M = U^T Gb F^T U diag(1/s)
#pragma unroll
    for (int a = 0; a < 3; ++a)
#pragma unroll
      for (int b = 0; b < 3; ++b) T[3 * a + b] = Hob[3 * a] * F[3 * b] + Hob[3 * a + 1] * F[3 * b + 1] + Hob[3 * a + 2] * F[3 * b + 2];
    ut_a_w(P.U, T, P.U, M);
#pragma unroll
    for (int a = 0; a < 3; ++a)
#pragma unroll
      for (int b = 0; b < 3; ++b) M[3 * a + b] /= P.s[b];
    float K[9];
#pragma unroll
    for (int kk = 0; kk < 3; ++kk) {
      const float de = P.beta[kk] > kBetaMin ? 1.0f / P.s[kk] : 0.0f;
      float acc = 0.0f;
#pragma unroll
      for (int i = 0; i < 3; ++i) {
        const float dn = ((i == kk ? 1.0f : 0.0f) - n[i] * n[kk] - (1.0f / 3.0f)) / nh;
        acc += M[4 * i] * g[i] * ((1.0f / 3.0f) + m.cyl * dn);
      }
      K[4 * kk] = acc * de;
    }
    const int PI[3] = {0, 0, 1}, PJ[3] = {1, 2, 2};
#pragma unroll
    for (int r = 0; r < 3; ++r) {
      const int i = PI[r], j = PJ[r];
      // eps_i - eps_j = (b_i - b_j) lr / 2 and s_i - s_j = (b_i - b_j)/(s_i + s_j)
      const float lr = log1p_ratio(P.beta[i], P.beta[j]);
      const float R = 0.5f * lr * (P.s[i] + P.s[j]);
      const float z = k * 0.5f * (P.beta[i] - P.beta[j]) * lr;
      const float A = g[j] * k * R * expm1_ratio(z);
      const float B = (g[i] + g[j]) / (P.s[i] + P.s[j]);
      const float sym = 0.5f * (M[3 * i + j] + M[3 * j + i]);
      const float asy = 0.5f * (M[3 * i + j] - M[3 * j + i]);
      K[3 * i + j] = A * sym + B * asy;
      K[3 * j + i] = A * sym - B * asy;
    }
    // Fb = U K diag(1/s) U^T F
#pragma unroll
    for (int a = 0; a < 3; ++a)
#pragma unroll
      for (int b = 0; b < 3; ++b) K[3 * a + b] /= P.s[b];
    float W[9];
    matmul3(P.U, K, T);
#pragma unroll
    for (int a = 0; a < 3; ++a)
#pragma unroll
      for (int b = 0; b < 3; ++b) W[3 * a + b] = T[3 * a] * P.U[3 * b] + T[3 * a + 1] * P.U[3 * b + 1] + T[3 * a + 2] * P.U[3 * b + 2];
    matmul3(W, F, Htb);
  } else if (m.kind == MAT_FLUID) {
    // d(J^(1/3) I) = (J^(-2/3)/3) tr(.) cof(F)
    const float J = 1.0f + detm1(Ht);
    const float c = (Hob[0] + Hob[4] + Hob[8]) * cbrtf(J) / (3.0f * J);
    float F[9], K[9];
    f_of(Ht, F);
    cofactor3(F, K);
#pragma unroll
    for (int i = 0; i < 9; ++i) Htb[i] = c * K[i];
  } else {
#pragma unroll
    for (int i = 0; i < 9; ++i) Htb[i] = Hob[i];
  }
}

// ------------------------------------------------------------------ colliders

enum { COLL_NONE = 0, COLL_CAPSULE = 1, COLL_BOX = 2, COLL_CONTAINER = 3, COLL_CAPSULES = 4 };

struct Coll {
  int kind;
  float dims[4];
  float mu, alpha;
};

// Length of the outside part (mx, my, mz) = max(q, 0) of a box SDF, rounded the same way
// wherever it is formed (the container compares these lengths between its boxes).
MPM_HD float box_outside_len(float mx, float my, float mz) {
  return sqrtf(__fmaf_rn(mz, mz, __fmaf_rn(my, my, __fmul_rn(mx, mx))));
}

// Signed distance of point p to the box of half extents h, alone: the d of sdf_box, bit for
// bit (outside: the length of max(q, 0); inside: the largest q).
MPM_HD float box_distance(float px, float py, float pz, float hx, float hy, float hz) {
  const float qx = fabsf(px) - hx, qy = fabsf(py) - hy, qz = fabsf(pz) - hz;
  if (qx > 0.0f || qy > 0.0f || qz > 0.0f) return box_outside_len(fmaxf(qx, 0.0f), fmaxf(qy, 0.0f), fmaxf(qz, 0.0f));
  return (qx >= qy && qx >= qz) ? qx : (qy >= qz ? qy : qz);
}

// Box SDF in its frame: d, gradient n, Hessian H (symmetric, 6 entries xx,xy,xz,yy,yz,zz).
MPM_HD void sdf_box(float px, float py, float pz, float hx, float hy, float hz, float& d, float* n, float* H) {
  float sx = px >= 0.0f ? 1.0f : -1.0f, sy = py >= 0.0f ? 1.0f : -1.0f, sz = pz >= 0.0f ? 1.0f : -1.0f;
  float qx = fabsf(px) - hx, qy = fabsf(py) - hy, qz = fabsf(pz) - hz;
  if (qx > 0.0f || qy > 0.0f || qz > 0.0f) {
    float mx = fmaxf(qx, 0.0f), my = fmaxf(qy, 0.0f), mz = fmaxf(qz, 0.0f);
    float l = box_outside_len(mx, my, mz);
    float r = 1.0f / l;
    d = l;
    n[0] = sx * mx * r; n[1] = sy * my * r; n[2] = sz * mz * r;
    H[0] = ((qx > 0.0f ? 1.0f : 0.0f) - n[0] * n[0]) * r;
    H[1] = -n[0] * n[1] * r;
    H[2] = -n[0] * n[2] * r;
    H[3] = ((qy > 0.0f ? 1.0f : 0.0f) - n[1] * n[1]) * r;
    H[4] = -n[1] * n[2] * r;
    H[5] = ((qz > 0.0f ? 1.0f : 0.0f) - n[2] * n[2]) * r;
  } else {
    n[0] = n[1] = n[2] = 0.0f;
    if (qx >= qy && qx >= qz) { d = qx; n[0] = sx; }
    else if (qy >= qz) { d = qy; n[1] = sy; }
    else { d = qz; n[2] = sz; }
#pragma unroll
    for (int i = 0; i < 6; ++i) H[i] = 0.0f;
  }
}

// Signed distance to the collider in its body frame: d, body-frame gradient nb and Hessian Hb.
MPM_HD void sdf_body(const Coll& c, float px, float py, float pz, float& d, float* nb, float* Hb) {
  if (c.kind == COLL_CAPSULE || c.kind == COLL_CAPSULES) {
    float R = c.dims[0], hl = c.dims[1];
    float ex = px - fminf(fmaxf(px, -hl), hl);
    float l = sqrtf(ex * ex + py * py + pz * pz);
    if (l < 1e-12f) {
      d = -R;
      nb[0] = 0.0f; nb[1] = 0.0f; nb[2] = 1.0f;
#pragma unroll
      for (int i = 0; i < 6; ++i) Hb[i] = 0.0f;
      return;
    }
    float r = 1.0f / l;
    d = l - R;
    nb[0] = ex * r; nb[1] = py * r; nb[2] = pz * r;
    float px_free = fabsf(px) < hl ? 0.0f : 1.0f;
    Hb[0] = (px_free - nb[0] * nb[0]) * r;
    Hb[1] = -nb[0] * nb[1] * r;
    Hb[2] = -nb[0] * nb[2] * r;
    Hb[3] = (1.0f - nb[1] * nb[1]) * r;
    Hb[4] = -nb[1] * nb[2] * r;
    Hb[5] = (1.0f - nb[2] * nb[2]) * r;
  } else if (c.kind == COLL_BOX) {
    sdf_box(px, py, pz, c.dims[0], c.dims[1], c.dims[2], d, nb, Hb);
  } else {
    // open-top container: floor and four walls; the walls reach down through the floor
    // (z in [-az - w, az]) and overlap at the vertical edges, so no two boxes share a face.
    // The nearest box (the first on a tie, floor first) gives d, its gradient and Hessian:
    // the five distances are compared alone, and only the chosen box is evaluated in full.
    const float a = c.dims[0], w = c.dims[1], az = c.dims[2];
    const float hw = 0.5f * w, hz = az + hw, ao = a + hw, aw = a + w;
    // the chosen box: the point in its frame (bx, by, bz) and its half extents (hx, hy, hzb)
    float bx = px, by = py, bz = pz + az + hw, hx = aw, hy = aw, hzb = hw;
    float best = box_distance(bx, by, bz, hx, hy, hzb);
#define MPM_WALL(OX, OY, HX, HY)                                   \
  {                                                                \
    const float wx = px - (OX), wy = py - (OY), wz = pz + hw;      \
    const float dk = box_distance(wx, wy, wz, HX, HY, hz);         \
    if (dk < best) {                                               \
      best = dk;                                                   \
      bx = wx; by = wy; bz = wz; hx = (HX); hy = (HY); hzb = hz;   \
    }                                                              \
  }
    MPM_WALL(ao, 0.0f, hw, aw)
    MPM_WALL(-ao, 0.0f, hw, aw)
    MPM_WALL(0.0f, ao, aw, hw)
    MPM_WALL(0.0f, -ao, aw, hw)
#undef MPM_WALL
    sdf_box(bx, by, bz, hx, hy, hzb, d, nb, Hb);
  }
}

struct Contact {
  float d;        // signed distance
  float n[3];     // world normal
  float H[6];     // world Hessian (symmetric)
  float dd_dth;   // dd/dtheta
  float dn_dth[3];
  float vb[3];    // body velocity at the node
};

// Collider at world point (x, y, z), pose q = (c, theta), pose velocity u = (v_c, omega);
// st, ct = sin theta, cos theta (the caller's, formed once for all nodes that share the pose).
template <bool kAdjoint>
MPM_HD void contact_eval(const Coll& c, float x, float y, float z, const float* q, const float* u, float st, float ct,
                         Contact& o) {
  float rx = x - q[0], ry = y - q[1], rz = z - q[2];
  float px = ct * rx + st * ry, py = -st * rx + ct * ry, pz = rz;  // R(-theta) r
  float nb[3], Hb[6];
  sdf_body(c, px, py, pz, o.d, nb, Hb);
  o.n[0] = ct * nb[0] - st * nb[1];
  o.n[1] = st * nb[0] + ct * nb[1];
  o.n[2] = nb[2];
  o.vb[0] = u[0] - u[3] * ry;
  o.vb[1] = u[1] + u[3] * rx;
  o.vb[2] = u[2];
  if (kAdjoint) {
    // H = R Hb R^T for a rotation about z
    float h00 = Hb[0], h01 = Hb[1], h02 = Hb[2], h11 = Hb[3], h12 = Hb[4], h22 = Hb[5];
    float a00 = ct * h00 - st * h01, a01 = ct * h01 - st * h11, a02 = ct * h02 - st * h12;  // row 0 of R Hb
    float a10 = st * h00 + ct * h01, a11 = st * h01 + ct * h11, a12 = st * h02 + ct * h12;  // row 1
    o.H[0] = a00 * ct - a01 * st;
    o.H[1] = a00 * st + a01 * ct;
    o.H[2] = a02;
    o.H[3] = a10 * st + a11 * ct;
    o.H[4] = a12;
    o.H[5] = h22;
    // dp/dtheta = (p_y, -p_x, 0)
    float tx = py, ty = -px;
    o.dd_dth = nb[0] * tx + nb[1] * ty;
    float hx = h00 * tx + h01 * ty, hy = h01 * tx + h11 * ty, hz = h02 * tx + h12 * ty;
    float kx = -nb[1] + hx, ky = nb[0] + hy;  // K nb + Hb tb (body frame)
    o.dn_dth[0] = ct * kx - st * ky;
    o.dn_dth[1] = st * kx + ct * ky;
    o.dn_dth[2] = hz;
  }
}

}  // namespace mpm
