// fem.cu -- tetrahedral-FEM environments (App. D.2: stable neo-Hookean elements, forces from
// the energy gradient, semi-implicit Euler; App. E SoftJumper: damping, per-element
// activations).
//
// A mesh of a few hundred vertices is far too small to fill the GPU one substep at a time, so
// one CTA runs a whole control step of one environment with the vertex state in shared memory:
// per substep, each element writes its four corner forces to shared memory, then each vertex
// sums the corners of its elements through an incidence list (no atomics, so results are
// deterministic) and integrates.  Global memory is touched only at the step's ends (and, in
// reverse, for the recomputed substep states).  The CTAs of all FEM environments run side by
// side.
//
// Per element e with vertices (i0..i3): Ds = [x_i1 - x_i0, x_i2 - x_i0, x_i3 - x_i0],
// F = Ds Dm^-1, J = det F, I_C = |F|^2, a = act_scale * action[group(e)],
//   P = mu (1 - 1/(I_C + 1)) F + lam (J - alpha - a) cof(F) + k_damp Fdot,  Fdot = Vs Dm^-1,
// forces f_{c+1} = -V0 (P Dm^-T)[:, c], f_0 = -sum_c f_{c+1}.  Vertices: w = v + dt (f / m + g);
// at or below the ground and moving down, w_z = 0 and w_t *= max(0, 1 + mu_g w_z / |w_t|);
// then v = w, x += dt w.  The reverse kernel is the exact adjoint of these steps.
//
// Within a control step each position is carried as an unevaluated FP32 sum hi + lo
// (compensated summation of the x += dt w updates): an update is a few 1e-5 of a position of
// order 0.5, so a plain FP32 sum would drop most of each update's low bits, and the elements'
// edge vectors, whose relative changes are the strain, would inherit that error.  The edge
// vectors are formed from the hi differences (exact for nearby vertices) plus the lo
// differences.  Positions are rounded to FP32 at control-step ends (the stored state).
#include <algorithm>

#include "kernels.h"
#include "mpm_types.h"

namespace mpm {

constexpr int kFemThreads = 256;

namespace {

struct FemLaw {
  float mu, lam, alpha, kd;
};

__device__ __forceinline__ void cross3(const float* a, const float* b, float* c) {
  c[0] = a[1] * b[2] - a[2] * b[1];
  c[1] = a[2] * b[0] - a[0] * b[2];
  c[2] = a[0] * b[1] - a[1] * b[0];
}

// cof(F) = dJ/dF: row r is the cross product of the other two rows (cyclic).
__device__ __forceinline__ void cofac(const float* F, float* C) {
  cross3(F + 3, F + 6, C);
  cross3(F + 6, F, C + 3);
  cross3(F, F + 3, C + 6);
}

// Element edge matrix from component-major shared vertex arrays P[k * ns + i].
__device__ __forceinline__ void edge_mat(const float* P, int ns, int4 t, float* D) {
  const int vi[3] = {t.y, t.z, t.w};
#pragma unroll
  for (int k = 0; k < 3; ++k) {
    const float p0 = P[k * ns + t.x];
#pragma unroll
    for (int c = 0; c < 3; ++c) D[3 * k + c] = P[k * ns + vi[c]] - p0;
  }
}

// Edge matrix of positions held as hi + lo: (hi_j - hi_0) + (lo_j - lo_0).
__device__ __forceinline__ void edge_mat_x(const float* X, const float* XL, int ns, int4 t, float* D) {
  const int vi[3] = {t.y, t.z, t.w};
#pragma unroll
  for (int k = 0; k < 3; ++k) {
    const float h0 = X[k * ns + t.x], l0 = XL[k * ns + t.x];
#pragma unroll
    for (int c = 0; c < 3; ++c)
      D[3 * k + c] = __fsub_rn(X[k * ns + vi[c]], h0) + __fsub_rn(XL[k * ns + vi[c]], l0);
  }
}

// hi + lo += d, keeping hi + lo an unevaluated sum with |lo| <= ulp(hi) / 2 (|d| << |hi|).
__device__ __forceinline__ void add_compensated(float& hi, float& lo, float d) {
  const float y = __fadd_rn(d, lo);
  const float t = __fadd_rn(hi, y);
  lo = __fsub_rn(y, __fsub_rn(t, hi));
  hi = t;
}

__device__ __forceinline__ void mul3(const float* A, const float* B, float* C) {  // C = A B
#pragma unroll
  for (int i = 0; i < 3; ++i)
#pragma unroll
    for (int j = 0; j < 3; ++j) C[3 * i + j] = A[3 * i] * B[j] + A[3 * i + 1] * B[3 + j] + A[3 * i + 2] * B[6 + j];
}

__device__ __forceinline__ void mul3bt(const float* A, const float* B, float* C) {  // C = A B^T
#pragma unroll
  for (int i = 0; i < 3; ++i)
#pragma unroll
    for (int j = 0; j < 3; ++j)
      C[3 * i + j] = A[3 * i] * B[3 * j] + A[3 * i + 1] * B[3 * j + 1] + A[3 * i + 2] * B[3 * j + 2];
}

// Elastic stress of the stable neo-Hookean law; returns J.
__device__ __forceinline__ float stress(const FemLaw& m, const float* F, float a, float* P) {
  float C[9];
  cofac(F, C);
  float ic = 0.f;
#pragma unroll
  for (int q = 0; q < 9; ++q) ic += F[q] * F[q];
  const float J = F[0] * C[0] + F[1] * C[1] + F[2] * C[2];
  const float c1 = m.mu * (1.0f - 1.0f / (ic + 1.0f)), c2 = m.lam * (J - m.alpha - a);
#pragma unroll
  for (int q = 0; q < 9; ++q) P[q] = c1 * F[q] + c2 * C[q];
  return J;
}

// Adjoint of the elastic stress (the energy's Hessian applied to Pb) and of the activation.
__device__ __forceinline__ void stress_adj(const FemLaw& m, const float* F, float a, const float* Pb, float* Fb,
                                           float* ab) {
  float C[9];
  cofac(F, C);
  float ic = 0.f, fp = 0.f, cp = 0.f;
#pragma unroll
  for (int q = 0; q < 9; ++q) {
    ic += F[q] * F[q];
    fp += F[q] * Pb[q];
    cp += C[q] * Pb[q];
  }
  const float J = F[0] * C[0] + F[1] * C[1] + F[2] * C[2];
  const float i1 = 1.0f / (ic + 1.0f);
  const float c1 = m.mu * (1.0f - i1), c3 = 2.0f * m.mu * fp * i1 * i1, c4 = m.lam * cp, c5 = m.lam * (J - m.alpha - a);
  // d cof[Pb]: row r = Pb_{r+1} x F_{r+2} + F_{r+1} x Pb_{r+2} (rows cyclic)
  float D[9], u[3], w[3];
#pragma unroll
  for (int r = 0; r < 3; ++r) {
    const int r1 = r == 2 ? 0 : r + 1, r2 = r == 0 ? 2 : r - 1;
    cross3(Pb + 3 * r1, F + 3 * r2, u);
    cross3(F + 3 * r1, Pb + 3 * r2, w);
#pragma unroll
    for (int k = 0; k < 3; ++k) D[3 * r + k] = u[k] + w[k];
  }
#pragma unroll
  for (int q = 0; q < 9; ++q) Fb[q] = c1 * Pb[q] + c3 * F[q] + c4 * C[q] + c5 * D[q];
  *ab = -m.lam * cp;
}

__device__ __forceinline__ FemLaw law_of(const EnvDesc& e) { return FemLaw{e.mu, e.lam, e.fem_alpha, e.k_damp}; }

__device__ __forceinline__ float elem_act(const EnvDesc& e, const float* act, int el) {
  return e.act_stress * act[e.n_coll_act + e.fem_group[el]];
}

// Corner terms of an element for the four vertices from the 3x3 edge-column terms M
// (row k = component, column c = edge c): vertex c+1 gets M[:, c], vertex 0 gets -sum_c M[:, c].
// Written component-major, T[(3 corner + k) nts + el], so the lanes of a warp (consecutive
// elements) store to consecutive banks.
__device__ __forceinline__ void put_corners(float* T, int nts, int el, const float* M, float scale) {
#pragma unroll
  for (int k = 0; k < 3; ++k) {
    float s = 0.f;
#pragma unroll
    for (int c = 0; c < 3; ++c) {
      const float v = scale * M[3 * k + c];
      T[(3 * (c + 1) + k) * nts + el] = v;
      s += v;
    }
    T[k * nts + el] = -s;
  }
}

// Sum of vertex i's corner terms (incidence entries 4 el + corner, in shared memory).
__device__ __forceinline__ void gather_corners(const float* T, int nts, const int* voff, const int* vinc, int i,
                                               float* out) {
  float a0 = 0.f, a1 = 0.f, a2 = 0.f;
  for (int j = voff[i]; j < voff[i + 1]; ++j) {
    const int el = vinc[j] >> 2, c = vinc[j] & 3;
    const float* t = T + 3 * c * nts + el;
    a0 += t[0];
    a1 += t[nts];
    a2 += t[2 * nts];
  }
  out[0] = a0;
  out[1] = a1;
  out[2] = a2;
}

// Corner forces of every element at (X + XL, V) into EF (element stride nts); J <= 0 sets
// status 4.
__device__ void element_forces(const EnvDesc& e, const FemLaw& m, const float* act, const float* X, const float* XL,
                               const float* V, int ns, int nts, float* EF, int& status) {
  for (int el = threadIdx.x; el < e.n_tets; el += blockDim.x) {
    const int4 t = e.fem_tet[el];
    const float* Dmi = e.fem_dminv + 9 * el;
    float Dm[9], Ds[9], F[9], P[9], H[9];
#pragma unroll
    for (int q = 0; q < 9; ++q) Dm[q] = Dmi[q];
    edge_mat_x(X, XL, ns, t, Ds);
    mul3(Ds, Dm, F);
    const float J = stress(m, F, elem_act(e, act, el), P);
    if (!(J > 0.0f)) status |= 4;
    if (m.kd != 0.0f) {
      float Vs[9], Fd[9];
      edge_mat(V, ns, t, Vs);
      mul3(Vs, Dm, Fd);
#pragma unroll
      for (int q = 0; q < 9; ++q) P[q] += m.kd * Fd[q];
    }
    mul3bt(P, Dm, H);  // f_{c+1} = -V0 H[:, c]
    put_corners(EF, nts, el, H, -e.fem_vol[el]);
  }
}

// The new velocity w of a vertex at height z, projected by the ground.
__device__ __forceinline__ bool on_ground(const EnvDesc& e, float z, const float* w) {
  return z <= e.ground_z && w[2] < 0.0f;
}

// Shared-memory layout of one environment's step (floats; ints share the 4-byte slots).
struct FemSmem {
  float *X, *XL, *V, *Fv, *XB, *VB, *EA, *EB, *ABE;
  int *voff, *vinc, *goff, *ginc;
};

__device__ FemSmem carve(float* sm, int ns, int nts, int gs, bool reverse) {
  FemSmem s;
  s.X = sm;
  s.XL = s.X + 3 * ns;
  s.V = s.XL + 3 * ns;
  s.Fv = s.V + 3 * ns;
  float* p = s.Fv + 3 * ns;
  if (reverse) {
    s.XB = p;
    s.VB = s.XB + 3 * ns;
    p = s.VB + 3 * ns;
  } else {
    s.XB = s.VB = nullptr;
  }
  s.EA = p;
  p += 12 * nts;
  if (reverse) {
    s.EB = p;
    p += 12 * nts;
    s.ABE = p;
    p += nts;
  } else {
    s.EB = s.ABE = nullptr;
  }
  s.voff = reinterpret_cast<int*>(p);
  s.vinc = s.voff + ns + 1;
  s.goff = s.vinc + 4 * nts;
  s.ginc = s.goff + gs + 1;
  return s;
}

__device__ void stage_incidence(const EnvDesc& e, const FemSmem& s, bool groups) {
  for (int i = threadIdx.x; i <= e.n; i += blockDim.x) s.voff[i] = e.fem_vinc_off[i];
  for (int j = threadIdx.x; j < 4 * e.n_tets; j += blockDim.x) s.vinc[j] = e.fem_vinc[j];
  if (groups) {
    const int ng = e.n_groups > 0 ? e.n_groups : 1;
    for (int g = threadIdx.x; g <= ng; g += blockDim.x) s.goff[g] = e.fem_ginc_off[g];
    for (int j = threadIdx.x; j < e.n_tets; j += blockDim.x) s.ginc[j] = e.fem_ginc[j];
  }
}

__device__ void fem_substep(const EnvDesc& e, const FemLaw& m, const float* act, const FemSmem& s, int ns, int nts,
                            int& status) {
  element_forces(e, m, act, s.X, s.XL, s.V, ns, nts, s.EA, status);
  __syncthreads();
  const float dt = e.dt;
  for (int i = threadIdx.x; i < e.n; i += blockDim.x) {
    const float im = e.fem_inv_mass[i];
    float f[3], w[3];
    gather_corners(s.EA, nts, s.voff, s.vinc, i, f);
#pragma unroll
    for (int k = 0; k < 3; ++k) w[k] = s.V[k * ns + i] + dt * (im * f[k] + e.gravity[k]);
    if (on_ground(e, s.X[2 * ns + i], w)) {
      const float L = sqrtf(w[0] * w[0] + w[1] * w[1]);
      const float g = L > 0.0f ? fmaxf(0.0f, 1.0f + e.ground_mu * w[2] / L) : 0.0f;
      w[0] *= g;
      w[1] *= g;
      w[2] = 0.0f;
    }
#pragma unroll
    for (int k = 0; k < 3; ++k) {
      s.V[k * ns + i] = w[k];
      add_compensated(s.X[k * ns + i], s.XL[k * ns + i], dt * w[k]);
      if (!isfinite(s.X[k * ns + i])) status |= 2;
    }
  }
  __syncthreads();
}

// x, v of a state block into shared memory; with XL, the positions' low parts too: from
// components 6..8 of the block (ring blocks of the reverse pass keep them there), or zero
// when with_lo is false (a stored state is plain FP32).
__device__ __forceinline__ void load_xv(const float* b, long long np, int nv, int ns, float* X, float* V,
                                        float* XL = nullptr, bool with_lo = false) {
  for (int i = threadIdx.x; i < nv; i += blockDim.x)
#pragma unroll
    for (int k = 0; k < 3; ++k) {
      X[k * ns + i] = b[k * np + i];
      V[k * ns + i] = b[(3 + k) * np + i];
      if (XL) XL[k * ns + i] = with_lo ? b[(6 + k) * np + i] : 0.0f;
    }
}

// x, v from shared memory into a state block: with XL and keep_lo, the hi parts as x and the
// low parts in components 6..8 (ring blocks); with XL alone, x rounded from hi + lo.
__device__ __forceinline__ void store_xv(float* b, long long np, int nv, int ns, const float* X, const float* V,
                                         const float* XL = nullptr, bool keep_lo = false) {
  for (int i = threadIdx.x; i < nv; i += blockDim.x)
#pragma unroll
    for (int k = 0; k < 3; ++k) {
      const float hi = X[k * ns + i];
      b[k * np + i] = (XL && !keep_lo) ? __fadd_rn(hi, XL[k * ns + i]) : hi;
      if (XL && keep_lo) b[(6 + k) * np + i] = XL[k * ns + i];
      b[(3 + k) * np + i] = V[k * ns + i];
    }
}

// One CTA per FEM environment: the running control step's S substeps, from slot live to slot
// next (x, v; C and H written as zero, the meta words copied).
__global__ void __launch_bounds__(kFemThreads) k_fem_forward(const EnvDesc* __restrict__ envs,
                                                             const int* __restrict__ list, int ns, int nts) {
  extern __shared__ float sm[];
  const EnvDesc& e = envs[list[blockIdx.x]];
  const EnvCtr c = *e.ctr;
  const long long np = e.n_pad;
  const int nv = e.n;
  const FemSmem s = carve(sm, ns, nts, 0, false);
  const float* src = e.slots + (long long)c.live * e.block;
  float* dst = e.slots + (long long)c.next * e.block;
  const float* act = e.act + (long long)c.live * e.A;
  load_xv(src, np, nv, ns, s.X, s.V, s.XL, false);
  stage_incidence(e, s, false);
  __syncthreads();
  const FemLaw m = law_of(e);
  int status = 0;
  for (int k = 0; k < e.S; ++k) fem_substep(e, m, act, s, ns, nts, status);
  store_xv(dst, np, nv, ns, s.X, s.V, s.XL, false);
  for (int i = threadIdx.x; i < nv; i += blockDim.x) {
#pragma unroll
    for (int q = 6; q < kComp; ++q) dst[q * np + i] = 0.0f;
    reinterpret_cast<unsigned*>(dst + kComp * np)[i] = reinterpret_cast<const unsigned*>(src + kComp * np)[i];
  }
  status = __reduce_or_sync(0xffffffffu, status);
  if (status && (threadIdx.x & 31) == 0) atomicOr(&e.ctr->status, status);
}

// One CTA per FEM environment: the reverse of the step being reversed.  The substep states
// 1..S-1 are recomputed from the step's checkpoint into the ring, then the substeps are
// reversed last to first; the adjoint of the step's start state goes to the other adjoint
// buffer (the reverse step's end flips the parity), the activations' adjoints to the action
// accumulators.
__global__ void __launch_bounds__(kFemThreads) k_fem_reverse(const EnvDesc* __restrict__ envs,
                                                             const int* __restrict__ list, int ns, int nts, int gs) {
  extern __shared__ float sm[];
  const EnvDesc& e = envs[list[blockIdx.x]];
  const EnvCtr c = *e.ctr;
  const long long np = e.n_pad;
  const int nv = e.n, S = e.S;
  const FemSmem s = carve(sm, ns, nts, gs, true);
  const int slot = c.base + c.rev;
  const float* src = e.slots + (long long)slot * e.block;
  const float* act = e.act + (long long)slot * e.A;
  const FemLaw m = law_of(e);
  int status = 0;
  // recompute substep states 1..S-1 into ring blocks 0..S-2 (positions as hi and lo)
  load_xv(src, np, nv, ns, s.X, s.V, s.XL, false);
  stage_incidence(e, s, true);
  for (int el = threadIdx.x; el < e.n_tets; el += blockDim.x) s.ABE[el] = 0.0f;
  __syncthreads();
  for (int k = 0; k + 1 < S; ++k) {
    fem_substep(e, m, act, s, ns, nts, status);
    store_xv(e.ring + (long long)k * e.block, np, nv, ns, s.X, s.V, s.XL, true);
  }
  const float* adj = c.par ? e.adj1 : e.adj0;
  float* adj_out = c.par ? e.adj0 : e.adj1;
  load_xv(adj, np, nv, ns, s.XB, s.VB);
  const float dt = e.dt;
  for (int k = S - 1; k >= 0; --k) {
    // every thread reads back the ring vertices it wrote itself
    load_xv(k == 0 ? src : e.ring + (long long)(k - 1) * e.block, np, nv, ns, s.X, s.V, s.XL, k > 0);
    __syncthreads();
    element_forces(e, m, act, s.X, s.XL, s.V, ns, nts, s.EA, status);
    __syncthreads();
    // vertices: x' = x + dt w passes x-bar through and adds dt x-bar to w-bar; the ground
    // projection; w = v + dt (f / m + g) gives v-bar = w-bar and f-bar = dt w-bar / m
    for (int i = threadIdx.x; i < nv; i += blockDim.x) {
      const float im = e.fem_inv_mass[i];
      float f[3], w[3], ob[3], wb[3];
      gather_corners(s.EA, nts, s.voff, s.vinc, i, f);
#pragma unroll
      for (int k2 = 0; k2 < 3; ++k2) {
        w[k2] = s.V[k2 * ns + i] + dt * (im * f[k2] + e.gravity[k2]);
        ob[k2] = s.VB[k2 * ns + i] + dt * s.XB[k2 * ns + i];
        wb[k2] = ob[k2];
      }
      if (on_ground(e, s.X[2 * ns + i], w)) {
        const float L = sqrtf(w[0] * w[0] + w[1] * w[1]);
        const float g = L > 0.0f ? fmaxf(0.0f, 1.0f + e.ground_mu * w[2] / L) : 0.0f;
        if (L > 0.0f && g > 0.0f) {
          const float dot = ob[0] * w[0] + ob[1] * w[1];
          const float iL3 = 1.0f / (L * L * L);
          wb[0] = g * ob[0] - dot * e.ground_mu * w[2] * w[0] * iL3;
          wb[1] = g * ob[1] - dot * e.ground_mu * w[2] * w[1] * iL3;
          wb[2] = dot * e.ground_mu / L;
        } else {
          wb[0] = wb[1] = wb[2] = 0.0f;
        }
      }
#pragma unroll
      for (int k2 = 0; k2 < 3; ++k2) {
        s.VB[k2 * ns + i] = wb[k2];
        s.Fv[k2 * ns + i] = dt * im * wb[k2];  // f-bar
      }
    }
    __syncthreads();
    // elements: H-bar columns f-bar_{c+1} - f-bar_0; P-bar = -V0 H-bar Dm^-1; F-bar by the
    // energy's Hessian; Fdot-bar = k_damp P-bar; Ds-bar = F-bar Dm^-T, Vs-bar = Fdot-bar Dm^-T
    for (int el = threadIdx.x; el < e.n_tets; el += blockDim.x) {
      const int4 t = e.fem_tet[el];
      const float* Dmi = e.fem_dminv + 9 * el;
      const int vi[3] = {t.y, t.z, t.w};
      float Dm[9], Hb[9], Pb[9], Ds[9], F[9], Fb[9], Db[9], ab;
#pragma unroll
      for (int q = 0; q < 9; ++q) Dm[q] = Dmi[q];
#pragma unroll
      for (int k2 = 0; k2 < 3; ++k2) {
        const float f0 = s.Fv[k2 * ns + t.x];
#pragma unroll
        for (int cc = 0; cc < 3; ++cc) Hb[3 * k2 + cc] = s.Fv[k2 * ns + vi[cc]] - f0;
      }
      mul3(Hb, Dm, Pb);
      const float nv0 = -e.fem_vol[el];
#pragma unroll
      for (int q = 0; q < 9; ++q) Pb[q] *= nv0;
      edge_mat_x(s.X, s.XL, ns, t, Ds);
      mul3(Ds, Dm, F);
      stress_adj(m, F, elem_act(e, act, el), Pb, Fb, &ab);
      s.ABE[el] += ab;
      mul3bt(Fb, Dm, Db);
      put_corners(s.EA, nts, el, Db, 1.0f);
      if (m.kd != 0.0f) {
        mul3bt(Pb, Dm, Db);
        put_corners(s.EB, nts, el, Db, m.kd);
      }
    }
    __syncthreads();
    for (int i = threadIdx.x; i < nv; i += blockDim.x) {
      float xa[3], va[3];
      gather_corners(s.EA, nts, s.voff, s.vinc, i, xa);
#pragma unroll
      for (int k2 = 0; k2 < 3; ++k2) s.XB[k2 * ns + i] += xa[k2];
      if (m.kd != 0.0f) {
        gather_corners(s.EB, nts, s.voff, s.vinc, i, va);
#pragma unroll
        for (int k2 = 0; k2 < 3; ++k2) s.VB[k2 * ns + i] += va[k2];
      }
    }
    __syncthreads();
  }
  store_xv(adj_out, np, nv, ns, s.XB, s.VB);
  for (int i = threadIdx.x; i < nv; i += blockDim.x)
#pragma unroll
    for (int q = 6; q < kComp; ++q) adj_out[q * np + i] = 0.0f;
  // activations: per group, its elements in a fixed order (this CTA is the only writer of its
  // environment's action accumulators during the launch)
  for (int g = threadIdx.x; g < e.n_groups; g += blockDim.x) {
    float a = 0.0f;
    for (int j = s.goff[g]; j < s.goff[g + 1]; ++j) a += s.ABE[s.ginc[j]];
    e.acc[ACC_ACT + e.n_coll_act + g] += e.act_stress * a;
  }
  (void)status;
}

size_t fem_smem(int ns, int nts, int gs, bool reverse) {
  const size_t floats = (reverse ? 18 : 12) * (size_t)ns + (reverse ? 25 : 12) * (size_t)nts;
  const size_t ints = (size_t)ns + 1 + 4 * (size_t)nts + (reverse ? (size_t)gs + 1 + nts : 0);
  return 4 * (floats + ints);
}

void set_smem_attr(const void* fn, size_t sm, size_t& attr) {
  if (sm > attr) {
    cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
    attr = sm;
  }
}

}  // namespace

void launch_fem_forward(const Launch& L, const int* list, int n, int nv_max, int nt_max) {
  if (n <= 0) return;
  const int ns = (nv_max + 31) / 32 * 32;
  const size_t sm = fem_smem(ns, nt_max, 0, false);
  static size_t attr = 48 * 1024;
  set_smem_attr((const void*)k_fem_forward, sm, attr);
  LaunchScope ls(KC_OTHER, L.stream);
  k_fem_forward<<<n, kFemThreads, sm, L.stream>>>(L.envs, list, ns, nt_max);
}

void launch_fem_reverse(const Launch& L, const int* list, int n, int nv_max, int act_max, int nt_max) {
  if (n <= 0) return;
  const int ns = (nv_max + 31) / 32 * 32;
  const int gs = std::max(act_max, 1);
  const size_t sm = fem_smem(ns, nt_max, gs, true);
  static size_t attr = 48 * 1024;
  set_smem_attr((const void*)k_fem_reverse, sm, attr);
  LaunchScope ls(KC_OTHER, L.stream);
  k_fem_reverse<<<n, kFemThreads, sm, L.stream>>>(L.envs, list, ns, nt_max, gs);
}

}  // namespace mpm
