// fem.cu -- tetrahedral-FEM environments (App. D.2: stable neo-Hookean elements, forces from
// the energy gradient, semi-implicit Euler; App. E SoftJumper: damping, per-element
// activations).
//
// A mesh of a few hundred vertices is far too small to fill the GPU one substep at a time, so
// one CTA runs a whole control step of one environment with the vertex state in shared memory:
// per substep, the elements add their forces into a shared force array (shared atomics), then
// the vertices integrate.  Global memory is touched only at the step's ends (and, in reverse,
// for the recomputed substep states).  The CTAs of all FEM environments run side by side.
//
// Per element e with vertices (i0..i3): Ds = [x_i1 - x_i0, x_i2 - x_i0, x_i3 - x_i0],
// F = Ds Dm^-1, J = det F, I_C = |F|^2, a = act_scale * action[group(e)],
//   P = mu (1 - 1/(I_C + 1)) F + lam (J - alpha - a) cof(F) + k_damp Fdot,  Fdot = Vs Dm^-1,
// forces f_{c+1} = -V0 (P Dm^-T)[:, c], f_0 = -sum_c f_{c+1}.  Vertices: w = v + dt (f / m + g);
// at or below the ground and moving down, w_z = 0 and w_t *= max(0, 1 + mu_g w_z / |w_t|);
// then v = w, x += dt w.  The reverse kernel is the exact adjoint of these steps.
#include <algorithm>

#include "kernels.h"
#include "mpm_types.h"

namespace mpm {

constexpr int kFemThreads = 256;
constexpr int kFemStageElems = 1024;  // meshes up to this many elements keep them in shared memory

namespace {

struct FemLaw {
  float mu, lam, alpha, kd;
};

// Element data as the substeps read it: in shared memory (staged once per control step, with
// the step's activation per element) for meshes of up to kFemStageElems elements, else the
// environment's global arrays and the activation from the action vector.
struct Elems {
  const int4* tet;
  const float* dminv;
  const float* vol;
  const float* a;  // per-element activation, or NULL: act_scale * act[group]
  const int* group;
  const float* act;
  float act_scale;
  __device__ __forceinline__ float act_of(int el) const { return a ? a[el] : act_scale * act[group[el]]; }
};

// Shared-memory bytes reserved for staged element data when the largest mesh of a launch has
// nt_max elements: every mesh of up to kFemStageElems elements then fits.
__host__ __device__ __forceinline__ size_t stage_bytes(int nt_max) {
  return (size_t)(nt_max < kFemStageElems ? nt_max : kFemStageElems) * (16 + 36 + 4 + 4);
}

// Stage (when it fits) the element data behind `base` (16-byte aligned shared memory).
__device__ Elems stage_elems(const EnvDesc& e, const float* act, char* base) {
  const int nt = e.n_tets;
  const float* actv = act + e.n_coll_act;
  if (nt > kFemStageElems) return Elems{e.fem_tet, e.fem_dminv, e.fem_vol, nullptr, e.fem_group, actv, e.act_stress};
  int4* tet = reinterpret_cast<int4*>(base);
  float* dmi = reinterpret_cast<float*>(tet + nt);
  float* vol = dmi + 9 * nt;
  float* a = vol + nt;
  for (int el = threadIdx.x; el < nt; el += blockDim.x) {
    tet[el] = e.fem_tet[el];
    vol[el] = e.fem_vol[el];
    a[el] = e.act_stress * actv[e.fem_group[el]];
  }
  for (int q = threadIdx.x; q < 9 * nt; q += blockDim.x) dmi[q] = e.fem_dminv[q];
  return Elems{tet, dmi, vol, a, e.fem_group, actv, e.act_stress};
}

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

// Forces of every element at (X, V) into Fo (zeroed by the caller); J <= 0 sets status 4.
__device__ void element_forces(const EnvDesc& e, const FemLaw& m, const Elems& E, const float* X, const float* V,
                               float* Fo, int ns, int& status) {
  for (int el = threadIdx.x; el < e.n_tets; el += blockDim.x) {
    const int4 t = E.tet[el];
    const float* Dmi = E.dminv + 9 * el;
    float Dm[9], Ds[9], F[9], P[9], H[9];
#pragma unroll
    for (int q = 0; q < 9; ++q) Dm[q] = Dmi[q];
    edge_mat(X, ns, t, Ds);
    mul3(Ds, Dm, F);
    const float J = stress(m, F, E.act_of(el), P);
    if (!(J > 0.0f)) status |= 4;
    if (m.kd != 0.0f) {
      float Vs[9], Fd[9];
      edge_mat(V, ns, t, Vs);
      mul3(Vs, Dm, Fd);
#pragma unroll
      for (int q = 0; q < 9; ++q) P[q] += m.kd * Fd[q];
    }
    mul3bt(P, Dm, H);
    const float nv0 = -E.vol[el];
    const int vi[3] = {t.y, t.z, t.w};
#pragma unroll
    for (int k = 0; k < 3; ++k) {
      float s = 0.f;
#pragma unroll
      for (int c = 0; c < 3; ++c) {
        const float f = nv0 * H[3 * k + c];
        atomicAdd(&Fo[k * ns + vi[c]], f);
        s += f;
      }
      atomicAdd(&Fo[k * ns + t.x], -s);
    }
  }
}

// Ground projection of the new velocity w of a vertex at height z.
__device__ __forceinline__ bool on_ground(const EnvDesc& e, float z, const float* w) {
  return z <= e.ground_z && w[2] < 0.0f;
}

__device__ void fem_substep(const EnvDesc& e, const FemLaw& m, const Elems& E, float* X, float* V, float* Fo, int ns,
                            int& status) {
  const int nv = e.n;
  for (int q = threadIdx.x; q < 3 * ns; q += blockDim.x) Fo[q] = 0.f;
  __syncthreads();
  element_forces(e, m, E, X, V, Fo, ns, status);
  __syncthreads();
  const float dt = e.dt;
  for (int i = threadIdx.x; i < nv; i += blockDim.x) {
    const float im = e.fem_inv_mass[i];
    float w[3];
#pragma unroll
    for (int k = 0; k < 3; ++k) w[k] = V[k * ns + i] + dt * (im * Fo[k * ns + i] + e.gravity[k]);
    if (on_ground(e, X[2 * ns + i], w)) {
      const float L = sqrtf(w[0] * w[0] + w[1] * w[1]);
      const float g = L > 0.0f ? fmaxf(0.0f, 1.0f + e.ground_mu * w[2] / L) : 0.0f;
      w[0] *= g;
      w[1] *= g;
      w[2] = 0.0f;
    }
#pragma unroll
    for (int k = 0; k < 3; ++k) {
      V[k * ns + i] = w[k];
      X[k * ns + i] += dt * w[k];
      if (!isfinite(X[k * ns + i])) status |= 2;
    }
  }
  __syncthreads();
}

__device__ __forceinline__ FemLaw law_of(const EnvDesc& e) { return FemLaw{e.mu, e.lam, e.fem_alpha, e.k_damp}; }

__device__ __forceinline__ void load_xv(const float* b, long long np, int nv, int ns, float* X, float* V) {
  for (int i = threadIdx.x; i < nv; i += blockDim.x)
#pragma unroll
    for (int k = 0; k < 3; ++k) {
      X[k * ns + i] = b[k * np + i];
      V[k * ns + i] = b[(3 + k) * np + i];
    }
}

__device__ __forceinline__ void store_xv(float* b, long long np, int nv, int ns, const float* X, const float* V) {
  for (int i = threadIdx.x; i < nv; i += blockDim.x)
#pragma unroll
    for (int k = 0; k < 3; ++k) {
      b[k * np + i] = X[k * ns + i];
      b[(3 + k) * np + i] = V[k * ns + i];
    }
}

// One CTA per FEM environment: the running control step's S substeps, from slot live to slot
// next (x, v; C and H written as zero, the meta words copied).
__global__ void __launch_bounds__(kFemThreads) k_fem_forward(const EnvDesc* __restrict__ envs,
                                                             const int* __restrict__ list, int ns) {
  extern __shared__ float sm[];
  const EnvDesc& e = envs[list[blockIdx.x]];
  const EnvCtr c = *e.ctr;
  const long long np = e.n_pad;
  const int nv = e.n;
  float *X = sm, *V = sm + 3 * ns, *Fo = sm + 6 * ns;
  const float* src = e.slots + (long long)c.live * e.block;
  float* dst = e.slots + (long long)c.next * e.block;
  const float* act = e.act + (long long)c.live * e.A;
  load_xv(src, np, nv, ns, X, V);
  const Elems E = stage_elems(e, act, reinterpret_cast<char*>(sm + 9 * ns));
  __syncthreads();
  const FemLaw m = law_of(e);
  int status = 0;
  for (int k = 0; k < e.S; ++k) fem_substep(e, m, E, X, V, Fo, ns, status);
  store_xv(dst, np, nv, ns, X, V);
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
                                                             const int* __restrict__ list, int ns, int a_stride) {
  extern __shared__ float sm[];
  const EnvDesc& e = envs[list[blockIdx.x]];
  const EnvCtr c = *e.ctr;
  const long long np = e.n_pad;
  const int nv = e.n, S = e.S;
  float *X = sm, *V = sm + 3 * ns, *Fo = sm + 6 * ns, *XB = sm + 9 * ns, *VB = sm + 12 * ns, *AB = sm + 15 * ns;
  // staged element data after AB (a_stride rounded up to 4 floats keeps it 16-byte aligned)
  const int slot = c.base + c.rev;
  const float* src = e.slots + (long long)slot * e.block;
  const float* act = e.act + (long long)slot * e.A;
  const FemLaw m = law_of(e);
  int status = 0;
  // recompute substep states 1..S-1 into ring blocks 0..S-2
  load_xv(src, np, nv, ns, X, V);
  for (int g = threadIdx.x; g < a_stride; g += blockDim.x) AB[g] = 0.0f;
  const Elems E = stage_elems(e, act, reinterpret_cast<char*>(AB + a_stride));
  __syncthreads();
  for (int k = 0; k + 1 < S; ++k) {
    fem_substep(e, m, E, X, V, Fo, ns, status);
    store_xv(e.ring + (long long)k * e.block, np, nv, ns, X, V);
  }
  const float* adj = c.par ? e.adj1 : e.adj0;
  float* adj_out = c.par ? e.adj0 : e.adj1;
  load_xv(adj, np, nv, ns, XB, VB);
  __syncthreads();  // ring writes of this CTA are read back below by the same threads' peers
  const float dt = e.dt;
  for (int k = S - 1; k >= 0; --k) {
    load_xv(k == 0 ? src : e.ring + (long long)(k - 1) * e.block, np, nv, ns, X, V);
    for (int q = threadIdx.x; q < 3 * ns; q += blockDim.x) Fo[q] = 0.f;
    __syncthreads();
    element_forces(e, m, E, X, V, Fo, ns, status);
    __syncthreads();
    // vertices: x' = x + dt w passes x-bar through and adds dt x-bar to w-bar; the ground
    // projection; w = v + dt (f / m + g) gives v-bar = w-bar and f-bar = dt w-bar / m
    for (int i = threadIdx.x; i < nv; i += blockDim.x) {
      const float im = e.fem_inv_mass[i];
      float w[3], ob[3], wb[3];
#pragma unroll
      for (int k2 = 0; k2 < 3; ++k2) {
        w[k2] = V[k2 * ns + i] + dt * (im * Fo[k2 * ns + i] + e.gravity[k2]);
        ob[k2] = VB[k2 * ns + i] + dt * XB[k2 * ns + i];
        wb[k2] = ob[k2];
      }
      if (on_ground(e, X[2 * ns + i], w)) {
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
        VB[k2 * ns + i] = wb[k2];
        Fo[k2 * ns + i] = dt * im * wb[k2];  // f-bar
      }
    }
    __syncthreads();
    // elements: H-bar columns f-bar_{c+1} - f-bar_0; P-bar = -V0 H-bar Dm^-1; F-bar by the
    // energy's Hessian; Fdot-bar = k_damp P-bar; Ds-bar = F-bar Dm^-T, Vs-bar = Fdot-bar Dm^-T
    for (int el = threadIdx.x; el < e.n_tets; el += blockDim.x) {
      const int4 t = E.tet[el];
      const float* Dmi = E.dminv + 9 * el;
      const int vi[3] = {t.y, t.z, t.w};
      float Dm[9], Hb[9], Pb[9], Ds[9], F[9], Fb[9], Db[9], ab;
#pragma unroll
      for (int q = 0; q < 9; ++q) Dm[q] = Dmi[q];
#pragma unroll
      for (int k2 = 0; k2 < 3; ++k2) {
        const float f0 = Fo[k2 * ns + t.x];
#pragma unroll
        for (int cc = 0; cc < 3; ++cc) Hb[3 * k2 + cc] = Fo[k2 * ns + vi[cc]] - f0;
      }
      mul3(Hb, Dm, Pb);
      const float nv0 = -E.vol[el];
#pragma unroll
      for (int q = 0; q < 9; ++q) Pb[q] *= nv0;
      edge_mat(X, ns, t, Ds);
      mul3(Ds, Dm, F);
      stress_adj(m, F, E.act_of(el), Pb, Fb, &ab);
      atomicAdd(&AB[e.fem_group[el]], ab);
      mul3bt(Fb, Dm, Db);
#pragma unroll
      for (int k2 = 0; k2 < 3; ++k2) {
        float s = 0.f;
#pragma unroll
        for (int cc = 0; cc < 3; ++cc) {
          atomicAdd(&XB[k2 * ns + vi[cc]], Db[3 * k2 + cc]);
          s += Db[3 * k2 + cc];
        }
        atomicAdd(&XB[k2 * ns + t.x], -s);
      }
      if (m.kd != 0.0f) {
#pragma unroll
        for (int q = 0; q < 9; ++q) Pb[q] *= m.kd;
        mul3bt(Pb, Dm, Db);
#pragma unroll
        for (int k2 = 0; k2 < 3; ++k2) {
          float s = 0.f;
#pragma unroll
          for (int cc = 0; cc < 3; ++cc) {
            atomicAdd(&VB[k2 * ns + vi[cc]], Db[3 * k2 + cc]);
            s += Db[3 * k2 + cc];
          }
          atomicAdd(&VB[k2 * ns + t.x], -s);
        }
      }
    }
    __syncthreads();
  }
  store_xv(adj_out, np, nv, ns, XB, VB);
  for (int i = threadIdx.x; i < nv; i += blockDim.x)
#pragma unroll
    for (int q = 6; q < kComp; ++q) adj_out[q * np + i] = 0.0f;
  for (int g = threadIdx.x; g < e.n_groups; g += blockDim.x)
    if (AB[g] != 0.0f) atomicAdd(e.acc + ACC_ACT + e.n_coll_act + g, e.act_stress * AB[g]);
  (void)status;
}

size_t fem_smem(int ns, int a_stride, int nt_max, bool reverse) {
  return sizeof(float) * (reverse ? (size_t)15 * ns + (size_t)a_stride : (size_t)9 * ns) + stage_bytes(nt_max);
}

}  // namespace

void launch_fem_forward(const Launch& L, const int* list, int n, int nv_max, int nt_max) {
  if (n <= 0) return;
  const int ns = (nv_max + 31) / 32 * 32;
  const size_t sm = fem_smem(ns, 0, nt_max, false);
  static size_t attr = 48 * 1024;
  if (sm > attr) {
    cudaFuncSetAttribute(k_fem_forward, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
    attr = sm;
  }
  LaunchScope ls(KC_OTHER, L.stream);
  k_fem_forward<<<n, kFemThreads, sm, L.stream>>>(L.envs, list, ns);
}

void launch_fem_reverse(const Launch& L, const int* list, int n, int nv_max, int act_max, int nt_max) {
  if (n <= 0) return;
  const int ns = (nv_max + 31) / 32 * 32;
  const int a_stride = (std::max(act_max, 1) + 3) / 4 * 4;
  const size_t sm = fem_smem(ns, a_stride, nt_max, true);
  static size_t attr = 48 * 1024;
  if (sm > attr) {
    cudaFuncSetAttribute(k_fem_reverse, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
    attr = sm;
  }
  LaunchScope ls(KC_OTHER, L.stream);
  k_fem_reverse<<<n, kFemThreads, sm, L.stream>>>(L.envs, list, ns, a_stride);
}

}  // namespace mpm
