// kernels.cu -- batched MLS-MPM substep kernels and their adjoints (sm_103a, FP32).
//
// One substep of every environment in a batch = three launches over all environments:
//   P2G  (App. D.3 CPIC step 2): one CTA per work item (a run of up to CHUNK particles of
//        one environment, consecutive in the binned order).  The CTA groups its particles
//        by cell, sums each cell's mass and momentum per stencil node in registers, adds the
//        sums to the dense grid with float4 atomics and marks the touched 4^3 tiles active
//        (appending them to a device list).
//   GRID (CPIC step 3): persistent warps over the active-tile list; node-local update
//        (p/m, gravity, softened SDF contact with friction, walls).
//   G2P  (CPIC step 4): one thread per particle; coalesced SoA reads, 27 float4 grid
//        gathers through L1, F update and plastic projection, coalesced SoA writes.
// The adjoint kernels mirror them: G2P^T scatters grid-velocity adjoints with P2G's
// grouped scheme, GRID^T is node-local and reduces the collider-pose adjoint per
// environment, P2G^T gathers grid adjoints per particle (Sec. 4.1 discrete adjoint).
#include <cuda_runtime.h>
#include <stdint.h>

#include <atomic>

#include "kernels.h"
#include "mpm_math.cuh"
#include "mpm_types.h"

namespace mpm {

constexpr int kBlock = 128;         // threads per particle CTA
constexpr int kPPT = 2;             // particles per thread

// ------------------------------------------------------------------ common device helpers

// Status bits of EnvCtr::status: 1 domain, 2 NaN/Inf, 4 inverted J, 8 a bounded wait on an
// asynchronous copy gave up.
constexpr int kStatusWait = 8;

// ---- bulk-asynchronous staging (TMA bulk copies) of contiguous particle-component runs
//
// One thread issues cp.async.bulk copies of a chunk's SoA component runs into shared memory;
// they complete on an mbarrier (transaction count = bytes), which every thread waits on.
// A copy needs 16-byte aligned source and destination and a size that is a multiple of 16
// bytes: chunks start at multiples of four particles, component arrays hold n_pad (a multiple
// of 32) floats, and a run of `count` particles is rounded up to four, which stays inside the
// array.  The wait is bounded: after kWaitLimit polls the caller sets kStatusWait, waits once
// more (again bounded) for copies still in flight into its shared memory, and skips the
// chunk's work.
constexpr int kWaitLimit = 1 << 22;

__device__ __forceinline__ unsigned smem_u32(const void* p) { return (unsigned)__cvta_generic_to_shared(p); }

__device__ __forceinline__ void mbar_init(unsigned long long* bar, unsigned count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(bar)), "r"(count) : "memory");
  asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
}

// The calling thread's arrival, announcing `bytes` of copies that complete on the barrier.
__device__ __forceinline__ void mbar_arrive_expect_tx(unsigned long long* bar, unsigned bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(bar)), "r"(bytes) : "memory");
}

__device__ __forceinline__ void bulk_copy_g2s(void* dst, const void* src, unsigned bytes, unsigned long long* bar) {
  asm volatile("cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];"
               ::"r"(smem_u32(dst)), "l"(src), "r"(bytes), "r"(smem_u32(bar)) : "memory");
}

// Waits for the barrier's phase `parity` to complete; false after `limit` polls.
__device__ __forceinline__ bool mbar_wait(unsigned long long* bar, unsigned parity, int limit = kWaitLimit) {
  for (int it = 0; it < limit; ++it) {
    unsigned done;
    asm volatile(
        "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n selp.u32 %0, 1, 0, p;\n}"
        : "=r"(done) : "r"(smem_u32(bar)), "r"(parity) : "memory");
    if (done) return true;
  }
  return false;
}

// Bytes of one staged component run of `count` particles (rounded up to four particles).
__device__ __forceinline__ unsigned run_bytes(int count) { return (unsigned)((count + 3) & ~3) * 4u; }

// Whether a chunk can be staged: read in place (no permutation), starting on a 16-byte
// boundary, and no longer than the stage.
__device__ __forceinline__ bool stageable(const WorkItem& it, const unsigned* perm) {
  return perm == nullptr && (it.start & 3) == 0 && it.count > 0 && it.count <= kBlock * kPPT;
}

// One thread: copy components comps[0..n) of particles [start, start + count) of the SoA
// block src (component stride np) into dst[0..n), completing on bar.  The caller has armed
// bar with the bytes of all its runs (mbar_arrive_expect_tx).
template <int kStride>
__device__ __forceinline__ void copy_runs(float (*dst)[kStride], const float* src, long long np, const int* comps,
                                          int n, int start, unsigned bytes, unsigned long long* bar) {
  for (int q = 0; q < n; ++q) bulk_copy_g2s(dst[q], src + comps[q] * np + start, bytes, bar);
}

__device__ __forceinline__ void load_env(const EnvDesc* envs, int env, EnvDesc& s, EnvCtr& c) {
  const int* src = reinterpret_cast<const int*>(envs + env);
  int* dst = reinterpret_cast<int*>(&s);
  constexpr int W = (int)(sizeof(EnvDesc) / 4);
  for (int i = threadIdx.x; i < W; i += blockDim.x) dst[i] = src[i];
  __syncthreads();
  if (threadIdx.x < 8) reinterpret_cast<int*>(&c)[threadIdx.x] = reinterpret_cast<const int*>(s.ctr)[threadIdx.x];
  __syncthreads();
}

__device__ __forceinline__ int ref_slot(const EnvCtr& c, int kind) {
  switch (kind) {
    case REF_LIVE: return c.live;
    case REF_NEXT: return c.next;
    case REF_REV: return c.base + c.rev;
    case REF_REVEND: return c.base + c.rev + 1;
    default: return 0;
  }
}

// Whether the step being reversed had its substep states kept by the forward pass: the last
// keep_n recorded steps did (the reverse pass leaves live at base + T).
__device__ __forceinline__ bool rev_kept(const EnvDesc& e, const EnvCtr& c) {
  return e.keep_n > 0 && c.live - c.base - c.rev <= e.keep_n;
}

__device__ __forceinline__ float* ref_block(const EnvDesc& e, const EnvCtr& c, StateRef r) {
  if (r.kind == REF_RING) return e.ring + (long long)(r.k - 1) * e.block;
  if (r.kind == REF_FWDK) {
    if (r.k == 0) return e.slots + (long long)c.live * e.block;
    if (r.k >= e.S || e.keep_n == 0) return e.slots + (long long)c.next * e.block;
    const int m = (c.live - c.base) % e.keep_n;
    return e.keep + ((long long)m * (e.S - 1) + (r.k - 1)) * e.block;
  }
  if (r.kind == REF_REVK) {
    if (r.k == 0) return e.slots + (long long)(c.base + c.rev) * e.block;
    if (r.k >= e.S) return e.slots + (long long)(c.base + c.rev + 1) * e.block;
    if (rev_kept(e, c)) return e.keep + ((long long)(c.rev % e.keep_n) * (e.S - 1) + (r.k - 1)) * e.block;
    return e.ring + (long long)(r.k - 1) * e.block;
  }
  return e.slots + (long long)ref_slot(c, r.kind) * e.block;
}

// The blocks of two state references, resolved by one thread and published in shared memory
// by the caller's next barrier (G2P: resolved in every thread, the resolution's branches cost
// it 72 bytes of spills; out of line in this one thread they cost nothing).
__device__ __noinline__ void resolve_refs(const EnvDesc& s, const EnvCtr& c, StateRef r0, StateRef r1, float** blk) {
  blk[0] = ref_block(s, c, r0);
  blk[1] = ref_block(s, c, r1);
}

// slot whose pose / actions / permutation belong to the running control step
__device__ __forceinline__ int step_slot(const EnvCtr& c, int rev) { return rev ? c.base + c.rev : c.live; }

__device__ __forceinline__ Mat env_mat(const EnvDesc& e) {
  Mat m;
  m.kind = e.material;
  m.mu = e.mu;
  m.lam = e.lam;
  m.cyl = e.cyl;
  m.bulk = e.bulk;
  m.visc = e.visc;
  m.act = e.act_stress;
  return m;
}

__device__ __forceinline__ float group_act(const EnvDesc& e, int slot, unsigned meta) {
  if (e.material != MAT_MUSCLE) return 0.0f;
  int g = (int)(meta >> 20) - 1;
  if (g < 0 || g >= e.n_groups) return 0.0f;
  return e.act[(long long)slot * e.A + e.n_coll_act + g];
}

__device__ __forceinline__ void load_state(const float* b, long long np, int j, float* s /*24*/) {
#pragma unroll
  for (int c = 0; c < kComp; ++c) s[c] = b[c * np + j];
}

// Bounding box of a CTA's particle stencils (nodes lx.. lx+nx-1, ...); its cells index the
// scatter's counting sort.
struct Box {
  int lx, ly, lz, nx, ny, nz;
};

// Block-wide min/max of the particles' base cells -> box of their stencils (base..base+2).
__device__ __forceinline__ Box make_box(const int (*base)[3], const bool* valid, int* sred /*6 ints smem*/) {
  int mn[3] = {1 << 30, 1 << 30, 1 << 30}, mx[3] = {-1, -1, -1};
#pragma unroll
  for (int p = 0; p < kPPT; ++p)
    if (valid[p]) {
#pragma unroll
      for (int k = 0; k < 3; ++k) {
        mn[k] = min(mn[k], base[p][k]);
        mx[k] = max(mx[k], base[p][k]);
      }
    }
  if (threadIdx.x < 6) sred[threadIdx.x] = threadIdx.x < 3 ? (1 << 30) : -1;
  __syncthreads();
#pragma unroll
  for (int k = 0; k < 3; ++k) {
    int a = __reduce_min_sync(0xffffffffu, mn[k]);
    int b = __reduce_max_sync(0xffffffffu, mx[k]);
    if ((threadIdx.x & 31) == 0) {
      atomicMin(&sred[k], a);
      atomicMax(&sred[3 + k], b);
    }
  }
  __syncthreads();
  Box bx;
  bx.lx = sred[0];
  bx.ly = sred[1];
  bx.lz = sred[2];
  bx.nx = sred[3] - sred[0] + 3;
  bx.ny = sred[4] - sred[1] + 3;
  bx.nz = sred[5] - sred[2] + 3;
  return bx;
}

__device__ __forceinline__ void mark_tile(const EnvDesc& e, int env, int ix, int iy, int iz, uint2* active,
                                          int* active_n) {
  int TG = e.G >> 2;
  int t = ((iz >> 2) * TG + (iy >> 2)) * TG + (ix >> 2);
  unsigned* f = e.tile + t;
  if (*((volatile unsigned*)f) == 0u) {
    if (atomicExch(f, 1u) == 0u) {
      int s = atomicAdd(active_n, 1);
      active[s] = make_uint2((unsigned)env, (unsigned)t);
    }
  }
}

__device__ __forceinline__ unsigned cell_pack(int b0, int b1, int b2) {
  return (unsigned)b0 | ((unsigned)b1 << 10) | ((unsigned)b2 << 20);
}

// ------------------------------------------------------------------ grouped scatter
//
// P2G and G2P^T both add, for every particle p and every node i of its stencil,
//     w_ip (q_p + A_p r_ip)            (r_ip = x_i - x_p)
// (and w_ip m_p for P2G's mass).  A CTA does it for its chunk of binned particles group by
// group, a group being the chunk's particles of one cell base (found by a counting sort in
// shared memory; runs of equal cell base in binned order when the chunk's cells outnumber the
// sort's capacity).  (1) Every particle writes a record to shared memory.  (2) Work units
// (group, z offset c) sum the group's contributions to the nine nodes base + (0..2, 0..2, c)
// in registers and add them straight into the grid with float4 atomics: nine per unit, so a
// node receives one atomic per occupied cell of its stencil instead of one per particle.
// Groups are taken in cell order (ordering them by size to balance a warp's lanes cost more
// than it saved).  An earlier version added the units into a shared-memory box of the
// chunk's nodes and flushed the box to the grid; without the box the kernels need fewer
// barriers and less shared memory, and G2P^T keeps more L1 for its grid gather.

// Scatter shapes the kernels are built for, by the capacity (cells) of the chunk's counting
// sort: 256-particle chunks on four-warp CTAs sorting up to 512 or 1024 cells, or the same
// chunks split into four 64-particle CTAs of one warp each sorting up to 256 cells
// (kScBoxWarp), whose barriers are warp-wide only.  The autotuner picks one per material.  A
// 256-particle chunk of a dense body spans 40-150 cells, a 64-particle one 15-60.
constexpr int kScBoxSmall = 512;
constexpr int kScBoxLarge = 1024;
constexpr int kScBoxWarp = 256;
constexpr int kRec = 24;  // floats per particle record

// Threads per CTA of the scatter kernels built for a sort capacity.
template <int kScBox>
struct ScatterThreads {
  static constexpr int value = kScBox == kScBoxWarp ? 32 : kBlock;
};

template <int kScBox>
struct ScatterShared {
  static constexpr int NT = ScatterThreads<kScBox>::value;
  float4 rec[kRec / 4 * NT * kPPT];       // particle records (96 B each): quad j of particle l at
                                          // rec[j * NT * kPPT + l], so the lanes of a warp
                                          // reading different particles hit different banks
  unsigned cellcnt[kScBox];               // particles per cell of the chunk, then offsets
  unsigned key[NT * kPPT];                // packed cell base per particle (~0u: none)
  unsigned short gstart[NT * kPPT + 1];   // first particle of each group, then the end
  unsigned short sidx[NT * kPPT];         // grouped position -> particle record
  int seg[kPPT * NT / 32];                // group heads per (particle slot, warp)
};

// The part of work item `it0` that CTA `blockIdx.x` of a scatter kernel with NT threads takes:
// 256-particle items are split into 128 / NT consecutive parts.  Returns false for an empty part.
template <int NT>
__device__ __forceinline__ bool scatter_part(const WorkItem& it0, WorkItem& it) {
  constexpr int kParts = kBlock / NT;
  const int sub = kParts > 1 ? (int)(blockIdx.x % kParts) : 0;
  it = it0;
  it.start += sub * NT * kPPT;
  it.count = min(max(it0.count - sub * NT * kPPT, 0), NT * kPPT);
  return it.count > 0;
}

// G2P^T's record quads: (q0 q1 q2 gx) (gy gz wx0 wx1) (wx2 wy0 wy1 wy2) (wz0 wz1 wz2 A00)
// (A01 A02 A10 A11) (A12 A20 A21 A22), quad j at r[j * kRecStride] (r = rec + particle), with
// g = f dx the particle's offset from its base node.
template <int kRecStride>
__device__ __forceinline__ void write_record(float4* r, const float* q, const float* g, const float* wx,
                                             const float* wy, const float* wz, const float* A) {
  r[0] = make_float4(q[0], q[1], q[2], g[0]);
  r[kRecStride] = make_float4(g[1], g[2], wx[0], wx[1]);
  r[2 * kRecStride] = make_float4(wx[2], wy[0], wy[1], wy[2]);
  r[3 * kRecStride] = make_float4(wz[0], wz[1], wz[2], A[0]);
  r[4 * kRecStride] = make_float4(A[1], A[2], A[3], A[4]);
  r[5 * kRecStride] = make_float4(A[5], A[6], A[7], A[8]);
}

// P2G's record quads: (b0 b1 b2 wx0) (wx1 wx2 wy0 wy1) (wy2 wz0 wz1 wz2) (X0 X1 X2 Y0)
// (Y1 Y2 Z0 Z1) (Z2 - - -), with b = q - A g the value at the base node and X, Y, Z = dx times
// the columns of A: the value at node base + (a, b, c) is b + a X + b Y + c Z, which the unit
// loop builds by additions along the stencil.  (G2P^T keeps the record above: its register
// budget has no room for the extra products.)
template <int kRecStride>
__device__ __forceinline__ void write_record_affine(float4* r, const float* q, const float* g, const float* wx,
                                                    const float* wy, const float* wz, const float* A, float dx) {
  float bq[3];
#pragma unroll
  for (int c = 0; c < 3; ++c) bq[c] = q[c] - (A[3 * c] * g[0] + A[3 * c + 1] * g[1] + A[3 * c + 2] * g[2]);
  r[0] = make_float4(bq[0], bq[1], bq[2], wx[0]);
  r[kRecStride] = make_float4(wx[1], wx[2], wy[0], wy[1]);
  r[2 * kRecStride] = make_float4(wy[2], wz[0], wz[1], wz[2]);
  r[3 * kRecStride] = make_float4(dx * A[0], dx * A[3], dx * A[6], dx * A[1]);
  r[4 * kRecStride] = make_float4(dx * A[4], dx * A[7], dx * A[2], dx * A[5]);
  r[5 * kRecStride] = make_float4(dx * A[8], 0.f, 0.f, 0.f);
}

// Step (2), after make_box (whose barriers publish the records and keys).
// kMass: P2G (mass component m w, tiles marked active); else G2P^T (three components).
template <bool kMass, int kScBox>
__device__ __forceinline__ void scatter_groups(ScatterShared<kScBox>& sh, const EnvDesc& e, int env, int count,
                                               const bool* valid, const int (*base)[3], const int* sred,
                                               const Box& bx, float pm, float4* grid, uint2* active,
                                               int* active_n) {
  constexpr int NT = ScatterThreads<kScBox>::value;
  constexpr int kRecStride = NT * kPPT;
  const int cnx = bx.nx - 2, cny = bx.ny - 2;
  // the counting sort needs a counter per cell of the chunk's bounding box of cell bases
  const bool fits = sred[3] >= 0 && cnx * cny * (bx.nz - 2) <= kScBox;
  unsigned* cnt = sh.cellcnt;  // per cell: particles, then offsets
  if (fits) {
    const int cvol = cnx * cny * (bx.nz - 2);
    for (int q = threadIdx.x; q < cvol; q += NT) cnt[q] = 0u;
  }
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  int ngrp = 0;
  if (fits) {
    // groups = the cells of the chunk: a counting sort by cell base inside the CTA keeps a
    // cell's particles together however far the binned order has drifted since the last sort
    __syncthreads();
    const int cvol = cnx * cny * (bx.nz - 2);
    int ci[kPPT], rk[kPPT];
#pragma unroll
    for (int p = 0; p < kPPT; ++p) {
      ci[p] = 0;
      rk[p] = 0;
      if (valid[p]) {
        ci[p] = ((base[p][2] - bx.lz) * cny + (base[p][1] - bx.ly)) * cnx + (base[p][0] - bx.lx);
        rk[p] = (int)atomicAdd(&cnt[ci[p]], 1u);
      }
    }
    __syncthreads();
    // exclusive scan of (particles | non-empty << 16) over the cells: offsets and group numbers
    const int per = (cvol + NT - 1) / NT;
    const int c0 = threadIdx.x * per;
    unsigned loc = 0;
    for (int q = 0; q < per && c0 + q < cvol; ++q) {
      const unsigned n = cnt[c0 + q];
      loc += n | (n ? 1u << 16 : 0u);
    }
    unsigned incl = loc;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      const unsigned t = __shfl_up_sync(0xffffffffu, incl, o);
      if (lane >= o) incl += t;
    }
    if (lane == 31) sh.seg[warp] = (int)incl;
    __syncthreads();
    unsigned run = incl - loc;
    unsigned total = 0;
    for (int w = 0; w < NT / 32; ++w) {
      const unsigned t = (unsigned)sh.seg[w];
      if (w < warp) run += t;
      total += t;
    }
    for (int q = 0; q < per && c0 + q < cvol; ++q) {
      const unsigned n = cnt[c0 + q];
      cnt[c0 + q] = run;
      if (n) sh.gstart[run >> 16] = (unsigned short)(run & 0xffffu);
      run += n | (n ? 1u << 16 : 0u);
    }
    ngrp = (int)(total >> 16);
    __syncthreads();
#pragma unroll
    for (int p = 0; p < kPPT; ++p)
      if (valid[p]) sh.sidx[(cnt[ci[p]] & 0xffffu) + rk[p]] = (unsigned short)(threadIdx.x + p * NT);
  } else {
    // groups = runs of equal keys in chunk order, numbered by a scan over (slot, warp) segments
    unsigned heads[kPPT];
#pragma unroll
    for (int p = 0; p < kPPT; ++p) {
      const int l = threadIdx.x + p * NT;
      const bool h = valid[p] && (l == 0 || sh.key[l - 1] != sh.key[l]);
      heads[p] = __ballot_sync(0xffffffffu, h);
      if (lane == 0) sh.seg[p * (NT / 32) + warp] = __popc(heads[p]);
      sh.sidx[l] = (unsigned short)l;
    }
    __syncthreads();
#pragma unroll
    for (int p = 0; p < kPPT; ++p) {
      const int sg = p * (NT / 32) + warp;
      int off = 0;
      for (int q = 0; q < sg; ++q) off += sh.seg[q];
      if (heads[p] >> lane & 1u)
        sh.gstart[off + __popc(heads[p] & ((1u << lane) - 1u))] = (unsigned short)(threadIdx.x + p * NT);
    }
    for (int q = 0; q < kPPT * (NT / 32); ++q) ngrp += sh.seg[q];
  }
  if (threadIdx.x == 0) sh.gstart[ngrp] = (unsigned short)count;
  __syncthreads();
  const float dx = e.dx;
  // units: (group, z offset c), each summing the nine nodes base + (0..2, 0..2, c)
  const int nunits = ngrp * 3;
  for (int u = threadIdx.x; u < nunits; u += NT) {
    const int g = u / 3, oc = u - 3 * g;
    const int q0 = sh.gstart[g], q1 = sh.gstart[g + 1];
    const unsigned key = sh.key[sh.sidx[q0]];
    const int cx = (int)(key & 1023u), cy = (int)((key >> 10) & 1023u), cz = (int)(key >> 20);
    // P2G: one unit per group marks the tiles of the group's stencil (those of its corners)
    if (kMass && oc == 0)
      for (int mz = 0; mz < 3; mz += 2)
        for (int my = 0; my < 3; my += 2)
          for (int mx = 0; mx < 3; mx += 2) mark_tile(e, env, cx + mx, cy + my, cz + mz, active, active_n);
    float am[3][3], ap[3][3][3];
#pragma unroll
    for (int ob = 0; ob < 3; ++ob)
#pragma unroll
      for (int a = 0; a < 3; ++a) {
        am[ob][a] = 0.f;
        ap[ob][a][0] = ap[ob][a][1] = ap[ob][a][2] = 0.f;
      }
    if (kMass) {
      const float ocf = (float)oc;
      for (int q = q0; q < q1; ++q) {
        const float4* r = sh.rec + sh.sidx[q];
        const float4 r0 = r[0], r1 = r[kRecStride], r2 = r[2 * kRecStride], r3 = r[3 * kRecStride],
                     r4 = r[4 * kRecStride];
        const float z2 = reinterpret_cast<const float*>(r + 5 * kRecStride)[0];
        const float wzc = oc == 0 ? r2.y : (oc == 1 ? r2.z : r2.w);
        const float wya[3] = {r1.z, r1.w, r2.x};
        const float wxa[3] = {r0.w, r1.x, r1.y};
        // values along the stencil: b, plus c Z for the layer, b Y for the row, a X per node
        float t0 = r0.x + ocf * r4.z, t1 = r0.y + ocf * r4.w, t2 = r0.z + ocf * z2;
#pragma unroll
        for (int ob = 0; ob < 3; ++ob) {
          if (ob > 0) {
            t0 += r3.w;
            t1 += r4.x;
            t2 += r4.y;
          }
          const float wyz = wya[ob] * wzc;
          float u0 = t0, u1 = t1, u2 = t2;
#pragma unroll
          for (int a = 0; a < 3; ++a) {
            if (a > 0) {
              u0 += r3.x;
              u1 += r3.y;
              u2 += r3.z;
            }
            const float wt = wxa[a] * wyz;
            am[ob][a] += wt;
            ap[ob][a][0] += wt * u0;
            ap[ob][a][1] += wt * u1;
            ap[ob][a][2] += wt * u2;
          }
        }
      }
    } else {
      const float cdx = (float)oc * dx;
      for (int q = q0; q < q1; ++q) {
        const float4* r = sh.rec + sh.sidx[q];
        const float4 r0 = r[0], r1 = r[kRecStride], r2 = r[2 * kRecStride], r3 = r[3 * kRecStride],
                     r4 = r[4 * kRecStride], r5 = r[5 * kRecStride];
        const float wzc = oc == 0 ? r3.x : (oc == 1 ? r3.y : r3.z);
        const float rz = cdx - r1.y;
        const float tz0 = r0.x + r4.y * rz, tz1 = r0.y + r5.x * rz, tz2 = r0.z + r5.w * rz;
        const float wya[3] = {r2.y, r2.z, r2.w};
        const float wxa[3] = {r1.z, r1.w, r2.x};
        float rxa[3];
#pragma unroll
        for (int a = 0; a < 3; ++a) rxa[a] = (float)a * dx - r0.w;
#pragma unroll
        for (int ob = 0; ob < 3; ++ob) {
          const float ry = (float)ob * dx - r1.x;
          const float wyz = wya[ob] * wzc;
          const float t0 = tz0 + r4.x * ry, t1 = tz1 + r4.w * ry, t2 = tz2 + r5.z * ry;
#pragma unroll
          for (int a = 0; a < 3; ++a) {
            const float wt = wxa[a] * wyz;
            ap[ob][a][0] += wt * (t0 + r3.w * rxa[a]);
            ap[ob][a][1] += wt * (t1 + r4.z * rxa[a]);
            ap[ob][a][2] += wt * (t2 + r5.y * rxa[a]);
          }
        }
      }
    }
#pragma unroll
    for (int ob = 0; ob < 3; ++ob) {
      float4* gp = grid + ((long long)(cz + oc) * e.G + (cy + ob)) * e.G + cx;
#pragma unroll
      for (int a = 0; a < 3; ++a)
        atomicAdd(gp + a, kMass ? make_float4(am[ob][a] * pm, ap[ob][a][0], ap[ob][a][1], ap[ob][a][2])
                                : make_float4(ap[ob][a][0], ap[ob][a][1], ap[ob][a][2], 0.f));
    }
  }
}

// ------------------------------------------------------------------ P2G
//
// Grouped scatter of mass and APIC momentum (q = m v, A = m C - dt V D^-1 tau).

template <int MAT, int BOX>
__global__ void __launch_bounds__(ScatterThreads<BOX>::value, BOX == kScBoxWarp ? 20 : (BOX == kScBoxSmall ? 7 : 5))
    k_p2g(const EnvDesc* __restrict__ envs, const WorkItem* __restrict__ items, int item_off, StateRef src,
          int use_perm, int k, int rev, uint2* active, int* active_n, const int2* __restrict__ skip_slot,
          int tape_T, int tape_S) {
  constexpr int NT = ScatterThreads<BOX>::value;
  __shared__ EnvDesc e;
  __shared__ EnvCtr c;
  __shared__ int sred[6];
  __shared__ ScatterShared<BOX> sh;
  WorkItem it;
  if (!scatter_part<NT>(items[item_off + blockIdx.x / (kBlock / NT)], it)) return;
  // in the reverse pass, the grid tape restores this substep's grid when it was kept
  if (skip_slot != nullptr) {
    const int t = envs[it.env].ctr->rev;
    if (t >= 0 && t < tape_T && skip_slot[t * tape_S + k].y >= 0) return;
  }
  load_env(envs, it.env, e, c);
  const float* b = ref_block(e, c, src);
  const int sslot = step_slot(c, rev);
  const unsigned* perm = use_perm ? e.perm + (long long)sslot * e.n_pad : nullptr;
  const long long np = e.n_pad;
  const float G = (float)e.G;
  Mat m = env_mat(e);
  m.kind = MAT;  // compile-time material: the other laws' code is folded away
  const float Dinv = 4.0f * G * G;
  const float stress_k = -e.dt * e.p_vol * Dinv;
  const float pm = e.p_mass;
  const float dx = e.dx;
  int base[kPPT][3];
  bool valid[kPPT];
  int oob = 0;
#pragma unroll
  for (int p = 0; p < kPPT; ++p) {
    const int l = threadIdx.x + p * NT;
    valid[p] = l < it.count;
    sh.key[l] = 0xffffffffu;
    if (!valid[p]) continue;
    const int i = it.start + l;
    const int j = perm ? (int)perm[i] : i;
    float s[kComp];
    load_state(b, np, j, s);
#pragma unroll
    for (int a = 0; a < 3; ++a) base[p][a] = cell_base(s[a], G, e.G, &oob);
    sh.key[l] = cell_pack(base[p][0], base[p][1], base[p][2]);
    const unsigned meta = reinterpret_cast<const unsigned*>(b + kComp * np)[j];
    const float a_g = MAT == MAT_MUSCLE ? group_act(e, sslot, meta) : 0.0f;
    float tau[9];
    kirchhoff(m, s + 15, s + 6, a_g, tau);
    float A[9];
#pragma unroll
    for (int q = 0; q < 9; ++q) A[q] = pm * s[6 + q] + stress_k * tau[q];
    float wx[3], wy[3], wz[3], dw[3];
    const float f0 = __fmul_rn(s[0], G) - (float)base[p][0];
    const float f1 = __fmul_rn(s[1], G) - (float)base[p][1];
    const float f2 = __fmul_rn(s[2], G) - (float)base[p][2];
    bspline(f0, wx, dw);
    bspline(f1, wy, dw);
    bspline(f2, wz, dw);
    const float mv[3] = {pm * s[3], pm * s[4], pm * s[5]};
    const float g[3] = {f0 * dx, f1 * dx, f2 * dx};
    write_record_affine<NT * kPPT>(sh.rec + l, mv, g, wx, wy, wz, A, dx);
  }
  if (oob) atomicOr(&e.ctr->status, 1);
  const Box bx = make_box(base, valid, sred);
  scatter_groups<true, BOX>(sh, e, it.env, it.count, valid, base, sred, bx, pm, e.grid_mp, active, active_n);
}

// ------------------------------------------------------------------ grid update

struct NodeFwd {
  float v0[3], v1[3], v2[3], v3[3];
  float sc, vn, L, f, gL, gf;
  float vr[3], vt[3], vr2[3];
  float dl[3];  // vr2 - vr, evaluated without cancellation
  int branch, ground, which;
  unsigned zero;
  Contact ct;
};

// Forward node update; records the trace needed by its adjoint.
// Signed distance from world point (x, y, z) to a capsule (radius R, half length hl along the
// body x axis) at pose q, with st, ct = sin, cos of its angle q[3].
__device__ __forceinline__ float capsule_distance(float R, float hl, const float* q, float st, float ct, float x,
                                                  float y, float z) {
  const float rx = x - q[0], ry = y - q[1], rz = z - q[2];
  const float px = ct * rx + st * ry, py = -st * rx + ct * ry;
  const float ex = px - fminf(fmaxf(px, -hl), hl);
  return sqrtf(ex * ex + py * py + rz * rz) - R;
}

// Union of capsules: the nearest capsule to the node (smallest signed distance, the first on a
// tie) decides the contact.  q, u hold capsule 0's pose and velocity on entry and the chosen
// capsule's on return, sc = (sin, cos) of capsule 0's angle on entry and of the chosen one's
// on return; ps is the slot's pose vector, kdt the substep's time since the slot.
__device__ __forceinline__ int nearest_capsule(const EnvDesc& e, const float* ps, float kdt, float x, float y,
                                               float z, float* q, float* u, float* sc) {
  const float R = e.coll_dims[0], hl = e.coll_dims[1];
  float best = capsule_distance(R, hl, q, sc[0], sc[1], x, y, z);
  int which = 0;
  float bs = sc[0], bc = sc[1];
  for (int j = 1; j < e.n_caps; ++j) {
    float qj[4], sj, cj;
#pragma unroll
    for (int i = 0; i < 4; ++i) qj[i] = ps[4 * j + i] + kdt * e.acc[ACC_U + 4 * j + i];
    sincosf(qj[3], &sj, &cj);
    const float dj = capsule_distance(R, hl, qj, sj, cj, x, y, z);
    if (dj < best) {
      best = dj;
      which = j;
      bs = sj;
      bc = cj;
    }
  }
  if (which != 0) {
#pragma unroll
    for (int i = 0; i < 4; ++i) {
      u[i] = e.acc[ACC_U + 4 * which + i];
      q[i] = ps[4 * which + i] + kdt * u[i];
    }
    sc[0] = bs;
    sc[1] = bc;
  }
  return which;
}

// q, u: the collider pose and velocity (capsule 0 for the capsule union, replaced by the
// nearest capsule's, whose index is t.which); ps, kdt as for nearest_capsule; st0, ct0: sin and
// cos of q[3] on entry (the same for every node of the environment at this substep, so the
// callers form them once per tile).
template <bool kAdj>
__device__ __forceinline__ void node_forward(const EnvDesc& e, int ix, int iy, int iz, float4 mp, float* q, float* u,
                                             const float* ps, float kdt, float st0, float ct0, NodeFwd& t) {
  const float inv_m = 1.0f / mp.x;
  t.v0[0] = mp.y * inv_m;
  t.v0[1] = mp.z * inv_m;
  t.v0[2] = mp.w * inv_m;
#pragma unroll
  for (int i = 0; i < 3; ++i) t.v1[i] = t.v0[i] + e.dt * e.gravity[i];
#pragma unroll
  for (int i = 0; i < 3; ++i) t.v2[i] = t.v1[i];
  t.branch = 0;
  t.which = 0;
  if (e.coll_kind != COLL_NONE) {
    float sc[2] = {st0, ct0};
    if (e.coll_kind == COLL_CAPSULES) t.which = nearest_capsule(e, ps, kdt, ix * e.dx, iy * e.dx, iz * e.dx, q, u, sc);
    Coll cl;
    cl.kind = e.coll_kind;
#pragma unroll
    for (int i = 0; i < 4; ++i) cl.dims[i] = e.coll_dims[i];
    cl.mu = e.coll_mu;
    cl.alpha = e.alpha;
    contact_eval<kAdj>(cl, ix * e.dx, iy * e.dx, iz * e.dx, q, u, sc[0], sc[1], t.ct);
    t.sc = t.ct.d > 0.0f ? expf(-e.alpha * t.ct.d) : 1.0f;
#pragma unroll
    for (int i = 0; i < 3; ++i) t.vr[i] = t.v1[i] - t.ct.vb[i];
    t.vn = t.vr[0] * t.ct.n[0] + t.vr[1] * t.ct.n[1] + t.vr[2] * t.ct.n[2];
    // v2 = v1 + s (v_proj - v1) with v_proj = vr2 + vb, i.e. v1 + s (vr2 - vr).  The
    // difference dl = vr2 - vr is formed directly: 0 when separating, vn (mu vt/L - n)
    // when sliding, -vr when stopped.  (Adding vb back and subtracting v1 in FP32 would
    // leave an ulp of |vb| on every node the collider touches.)
    if (t.vn < 0.0f) {
#pragma unroll
      for (int i = 0; i < 3; ++i) t.vt[i] = t.vr[i] - t.vn * t.ct.n[i];
      t.L = sqrtf(t.vt[0] * t.vt[0] + t.vt[1] * t.vt[1] + t.vt[2] * t.vt[2]);
      t.f = t.L > 0.0f ? 1.0f + e.coll_mu * t.vn / t.L : 0.0f;
      if (t.f > 0.0f) {
        t.branch = 1;
        const float muL = e.coll_mu / t.L;
#pragma unroll
        for (int i = 0; i < 3; ++i) {
          t.vr2[i] = t.f * t.vt[i];
          t.dl[i] = t.vn * (muL * t.vt[i] - t.ct.n[i]);
        }
      } else {
        t.branch = 2;
#pragma unroll
        for (int i = 0; i < 3; ++i) {
          t.vr2[i] = 0.0f;
          t.dl[i] = -t.vr[i];
        }
      }
    } else {
#pragma unroll
      for (int i = 0; i < 3; ++i) {
        t.vr2[i] = t.vr[i];
        t.dl[i] = 0.0f;
      }
    }
#pragma unroll
    for (int i = 0; i < 3; ++i) t.v2[i] = t.v1[i] + t.sc * t.dl[i];
  }
#pragma unroll
  for (int i = 0; i < 3; ++i) t.v3[i] = t.v2[i];
  t.ground = 0;
  const int bnd = e.bound, G = e.G;
  if (iz < bnd && t.v2[2] < 0.0f) {
    t.ground = 1;
    if (e.ground_mu > 0.0f) {
      t.gL = sqrtf(t.v2[0] * t.v2[0] + t.v2[1] * t.v2[1]);
      t.gf = t.gL > 0.0f ? fmaxf(0.0f, 1.0f + e.ground_mu * t.v2[2] / t.gL) : 0.0f;
      t.v3[0] *= t.gf;
      t.v3[1] *= t.gf;
    }
    t.v3[2] = 0.0f;
  }
  t.zero = 0u;
  if ((ix < bnd && t.v3[0] < 0.0f) || (ix >= G - bnd && t.v3[0] > 0.0f)) t.zero |= 1u;
  if ((iy < bnd && t.v3[1] < 0.0f) || (iy >= G - bnd && t.v3[1] > 0.0f)) t.zero |= 2u;
  if (iz >= G - bnd && t.v3[2] > 0.0f) t.zero |= 4u;
}

// Pose vector of the running step's slot, and the pose (q, u) of body 0 at substep k.
__device__ __forceinline__ const float* step_pose(const EnvDesc& e, const EnvCtr& c, int rev, int k, float* q,
                                                  float* u) {
  const float* ps = e.pose + step_slot(c, rev) * kPose;
  const float kdt = (float)k * e.dt;
#pragma unroll
  for (int i = 0; i < 4; ++i) {
    u[i] = e.acc[ACC_U + i];
    q[i] = ps[i] + kdt * u[i];
  }
  return ps;
}

// Persistent warps over the active-tile list; one warp per 4^3 tile, two nodes per lane.
// Index of the recorded step running now (tape slot row), or -1 outside the tape.
__device__ __forceinline__ int tape_step_fwd(const EnvDesc* envs, int env0, const GridTape& tape) {
  const EnvCtr* c = envs[env0].ctr;
  const int t = c->live - c->base;
  return (t >= 0 && t < tape.T) ? t : -1;
}

// Index of the step being reversed, or -1 outside the tape.
__device__ __forceinline__ int tape_step_rev(const EnvDesc* envs, int env0, const GridTape& tape) {
  const int t = envs[env0].ctr->rev;
  return (t >= 0 && t < tape.T) ? t : -1;
}

// Recording (rec.mp set): the active tiles' (m, p) are also copied into the tape slot that
// k_tape_alloc reserved for this substep.
__global__ void __launch_bounds__(256, 3) k_grid(const EnvDesc* __restrict__ envs, const uint2* __restrict__ active,
                                                 const int* __restrict__ active_n, int k, int mode, int rev,
                                                 GridTape rec, int env0) {
  const int lane = threadIdx.x & 31;
  const int warp = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const int nwarps = (gridDim.x * blockDim.x) >> 5;
  const int n = *active_n;
  bool keep = false;
  long long first = 0;
  if (rec.mp != nullptr) {
    const int t = tape_step_fwd(envs, env0, rec);
    if (t >= 0) {
      const int2 sl = rec.slot[t * rec.S + k];
      keep = sl.y >= 0;
      first = sl.x;
    }
  }
  // A tile is a chain of dependent loads (list entry, descriptor, counters and pose, nodes):
  // the next tile's list entry is read one tile ahead, and a tile's two nodes per lane are
  // read before its counters and pose, so that those loads overlap.
  uint2 at_next = warp < n ? active[warp] : make_uint2(0u, 0u);
  for (int w = warp; w < n; w += nwarps) {
    const uint2 at = at_next;
    if (w + nwarps < n) at_next = active[w + nwarps];
    if (keep && lane == 0) rec.list[first + w] = at;
    const EnvDesc& e = envs[at.x];
    const int TG = e.G >> 2;
    const int tz = at.y / (TG * TG), ty = (at.y / TG) % TG, tx = at.y % TG;
    float4 mp[2];
#pragma unroll
    for (int h = 0; h < 2; ++h) {
      const int l = lane + 32 * h;
      const int ix = tx * 4 + (l & 3), iy = ty * 4 + ((l >> 2) & 3), iz = tz * 4 + (l >> 4);
      mp[h] = e.grid_mp[((long long)iz * e.G + iy) * e.G + ix];
    }
    const EnvCtr c = *e.ctr;
    float q0[4], u0[4];
    const float* ps = step_pose(e, c, rev, k, q0, u0);
    float st0, ct0;
    sincosf(q0[3], &st0, &ct0);
    const float kdt = (float)k * e.dt;
#pragma unroll
    for (int h = 0; h < 2; ++h) {
      const int l = lane + 32 * h;
      const int ix = tx * 4 + (l & 3), iy = ty * 4 + ((l >> 2) & 3), iz = tz * 4 + (l >> 4);
      const long long id = ((long long)iz * e.G + iy) * e.G + ix;
      if (keep) rec.mp[(first + w) * 64 + l] = mp[h];
      float4 out = make_float4(0.f, 0.f, 0.f, 0.f);
      if (mp[h].x > 0.0f) {
        NodeFwd t;
        float q[4] = {q0[0], q0[1], q0[2], q0[3]}, u[4] = {u0[0], u0[1], u0[2], u0[3]};
        node_forward<false>(e, ix, iy, iz, mp[h], q, u, ps, kdt, st0, ct0, t);
        out.x = (t.zero & 1u) ? 0.0f : t.v3[0];
        out.y = (t.zero & 2u) ? 0.0f : t.v3[1];
        out.z = (t.zero & 4u) ? 0.0f : t.v3[2];
      }
      e.grid_v[id] = out;
      if (mode == GRID_FWD) e.grid_mp[id] = make_float4(0.f, 0.f, 0.f, 0.f);
    }
    if (mode == GRID_FWD && lane == 0) e.tile[at.y] = 0u;
  }
}

// One thread: reserve the pool range of substep k of the recorded step (the first substep
// of the first recorded step starts the pool over).  A slot that does not fit is marked -1.
__global__ void k_tape_alloc(const EnvDesc* __restrict__ envs, int env0, GridTape tape, int k,
                             const int* __restrict__ active_n) {
  const int t = tape_step_fwd(envs, env0, tape);
  if (t < 0) return;
  if (t == 0 && k == 0) *tape.cursor = 0ull;
  const unsigned long long n = (unsigned long long)*active_n;
  const unsigned long long off = *tape.cursor;
  int2 sl = make_int2(0, -1);
  if (off + n <= (unsigned long long)tape.cap) {
    sl = make_int2((int)off, (int)n);
    *tape.cursor = off + n;
  }
  tape.slot[t * tape.S + k] = sl;
}

// Persistent warps over a kept slot of the step being reversed: (m, p) back into the dense
// grid, its tiles into the active list (which then holds exactly them).
__global__ void __launch_bounds__(256) k_restore(const EnvDesc* __restrict__ envs, int env0, GridTape tape, int k,
                                                 uint2* active, int* active_n) {
  const int t = tape_step_rev(envs, env0, tape);
  if (t < 0) return;
  const int2 sl = tape.slot[t * tape.S + k];
  const int n = sl.y;
  if (n < 0) return;
  if (blockIdx.x == 0 && threadIdx.x == 0) *active_n = n;
  const int lane = threadIdx.x & 31;
  const int warp = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const int nwarps = (gridDim.x * blockDim.x) >> 5;
  for (int w = warp; w < n; w += nwarps) {
    const uint2 at = tape.list[(long long)sl.x + w];
    if (lane == 0) active[w] = at;
    const EnvDesc& e = envs[at.x];
    const int TG = e.G >> 2;
    const int tz = at.y / (TG * TG), ty = (at.y / TG) % TG, tx = at.y % TG;
#pragma unroll
    for (int h = 0; h < 2; ++h) {
      const int l = lane + 32 * h;
      const int ix = tx * 4 + (l & 3), iy = ty * 4 + ((l >> 2) & 3), iz = tz * 4 + (l >> 4);
      e.grid_mp[((long long)iz * e.G + iy) * e.G + ix] = tape.mp[((long long)sl.x + w) * 64 + l];
    }
  }
}

// ------------------------------------------------------------------ G2P

template <int MAT>
// wait_polls: polls of the first wait on the staged copies (< 0: kWaitLimit); a test sets it
// to 0 to make that wait give up and exercise the status path.  use_stage: stage x and H by
// bulk copies when the chunk is read in place (the autotuner's choice).
__global__ void __launch_bounds__(kBlock, 8) k_g2p(const EnvDesc* __restrict__ envs, const WorkItem* __restrict__ items,
                                                int item_off, StateRef src, StateRef dst, int use_perm, int rev,
                                                int wait_polls, int use_stage) {
  __shared__ EnvDesc e;
  __shared__ EnvCtr c;
  // x and H of the chunk's particles, staged by bulk copies when they are read in place
  __shared__ alignas(16) float stage[12][kBlock * kPPT];
  __shared__ alignas(8) unsigned long long bar;
  const WorkItem it = items[item_off + blockIdx.x];
  if (threadIdx.x == 0) mbar_init(&bar, 1);
  __shared__ float* blk[2];
  load_env(envs, it.env, e, c);  // its barriers also publish the mbarrier's initialisation
  if (threadIdx.x == 0) resolve_refs(e, c, src, dst, blk);
  __syncthreads();
  const float* b = blk[0];
  float* o = blk[1];
  const int sslot = step_slot(c, rev);
  const unsigned* perm = use_perm ? e.perm + (long long)sslot * e.n_pad : nullptr;
  const long long np = e.n_pad;
  const bool staged = use_stage && stageable(it, perm);
  if (staged) {
    if (threadIdx.x == 0) {
      const int comps[12] = {0, 1, 2, 15, 16, 17, 18, 19, 20, 21, 22, 23};
      const unsigned bytes = run_bytes(it.count);
      mbar_arrive_expect_tx(&bar, 12 * bytes);
      copy_runs(stage, b, np, comps, 12, it.start, bytes, &bar);
    }
    // every thread polls on its own; the CTA leaves together if any of them gave up, thread 0
    // last, after a second bounded wait for the copies (its shared memory lives until then)
    if (!__syncthreads_and(mbar_wait(&bar, 0, wait_polls < 0 ? kWaitLimit : wait_polls) ? 1 : 0)) {
      if (threadIdx.x == 0) {
        atomicOr(&e.ctr->status, kStatusWait);
        (void)mbar_wait(&bar, 0);
      }
      return;
    }
  }
  const float G = (float)e.G;
  Mat m = env_mat(e);
  m.kind = MAT;  // compile-time material: the other laws' code is folded away
  const float Dinv = 4.0f * G * G, dt = e.dt, dx = e.dx;
  int status = 0;
#pragma unroll 1
  for (int p = 0; p < kPPT; ++p) {
    const int i = it.start + threadIdx.x + p * kBlock;
    if (i >= it.start + it.count) continue;
    const int j = perm ? (int)perm[i] : i;
    const int l = threadIdx.x + p * kBlock;
    float x[3];
#pragma unroll
    for (int a = 0; a < 3; ++a) x[a] = staged ? stage[a][l] : b[a * np + j];
    int base[3], oob = 0;
    float fx[3], w[3][3], dw[3];
#pragma unroll
    for (int a = 0; a < 3; ++a) {
      base[a] = cell_base(x[a], G, e.G, &oob);
      fx[a] = __fmul_rn(x[a], G) - (float)base[a];
      bspline(fx[a], w[a], dw);
    }
    if (oob) status |= 1;
    // With g_i = v_i - v_c (the stencil-centre velocity v_c adds v_c (sum w r)^T = 0 to C,
    // and subtracting it keeps the FP32 sums from cancelling):
    //   v = v_c sum w + sum w g,   C = D^-1 sum w g r^T.
    // The weights are separable, so each row of three nodes (y offset b, z offset c) is first
    // summed with w_x and w_x r_x, and the row's w_y w_z, r_y, r_z are applied once per row.
    const float4 vc = __ldg(e.grid_v + ((long long)(base[2] + 1) * e.G + (base[1] + 1)) * e.G + base[0] + 1);
    float wxr[3];
#pragma unroll
    for (int a = 0; a < 3; ++a) wxr[a] = w[0][a] * (((float)a - fx[0]) * dx);
    float sg[3] = {0.f, 0.f, 0.f}, C[9];
#pragma unroll
    for (int a = 0; a < 9; ++a) C[a] = 0.f;
#pragma unroll
    for (int cz = 0; cz < 3; ++cz) {
      const float rz = ((float)cz - fx[2]) * dx;
#pragma unroll
      for (int cy = 0; cy < 3; ++cy) {
        const float ry = ((float)cy - fx[1]) * dx;
        const float wyz = w[1][cy] * w[2][cz];
        const float4* row = e.grid_v + ((long long)(base[2] + cz) * e.G + (base[1] + cy)) * e.G + base[0];
        float s0[3] = {0.f, 0.f, 0.f}, s1[3] = {0.f, 0.f, 0.f};  // sum_a w_x g, sum_a w_x r_x g
#pragma unroll
        for (int cx = 0; cx < 3; ++cx) {
          const float4 nv = __ldg(row + cx);
          const float g0 = nv.x - vc.x, g1 = nv.y - vc.y, g2 = nv.z - vc.z;
          s0[0] += w[0][cx] * g0;
          s0[1] += w[0][cx] * g1;
          s0[2] += w[0][cx] * g2;
          s1[0] += wxr[cx] * g0;
          s1[1] += wxr[cx] * g1;
          s1[2] += wxr[cx] * g2;
        }
        const float wyr = wyz * ry, wzr = wyz * rz;
#pragma unroll
        for (int q = 0; q < 3; ++q) {
          sg[q] += wyz * s0[q];
          C[3 * q] += wyz * s1[q];
          C[3 * q + 1] += wyr * s0[q];
          C[3 * q + 2] += wzr * s0[q];
        }
      }
    }
    const float sw = (w[0][0] + w[0][1] + w[0][2]) * (w[1][0] + w[1][1] + w[1][2]) * (w[2][0] + w[2][1] + w[2][2]);
    const float v[3] = {vc.x * sw + sg[0], vc.y * sw + sg[1], vc.z * sw + sg[2]};
#pragma unroll
    for (int a = 0; a < 9; ++a) C[a] *= Dinv;
    // F <- (I + dt C) F, i.e. H <- H + dt (C + C H); then the plastic projection.  H is read
    // only now, so it is not held in registers through the stencil loop.
    float F[9];
#pragma unroll
    for (int a = 0; a < 9; ++a) F[a] = staged ? stage[3 + a][l] : b[(15 + a) * np + j];
    float CH[9], Ht[9], Fo[9];
    matmul3(C, F, CH);
#pragma unroll
    for (int a = 0; a < 9; ++a) Ht[a] = F[a] + dt * (C[a] + CH[a]);
    project(m, Ht, Fo);
    float xn[3];
#pragma unroll
    for (int a = 0; a < 3; ++a) {
      xn[a] = x[a] + dt * v[a];
      o[a * np + i] = xn[a];
      o[(3 + a) * np + i] = v[a];
      if (!isfinite(xn[a])) status |= 2;
    }
#pragma unroll
    for (int a = 0; a < 9; ++a) {
      o[(6 + a) * np + i] = C[a];
      o[(15 + a) * np + i] = Fo[a];
    }
    if (!(1.0f + detm1(Fo) > 0.0f)) status |= 4;
    if (perm || b != o) reinterpret_cast<unsigned*>(o + kComp * np)[i] = reinterpret_cast<const unsigned*>(b + kComp * np)[j];
  }
  status = __reduce_or_sync(0xffffffffu, status);
  if (status && (threadIdx.x & 31) == 0) atomicOr(&e.ctr->status, status);
}

// ------------------------------------------------------------------ step bookkeeping

// Pose velocity of a control step, u = act_scale * a / h: entry act_map[j] from action j, or
// for the capsule union entry j of capsule j / 4 from action j (scale act_scale[j % 4]).
__device__ __forceinline__ void pose_velocity(const EnvDesc& e, const float* a, float* u) {
  const float h = e.S * e.dt;
  if (e.coll_kind == COLL_CAPSULES) {
    for (int j = 0; j < 4 * e.n_caps; ++j) u[j] = e.act_scale[j & 3] * a[j] / h;
    return;
  }
  float w[4] = {0.f, 0.f, 0.f, 0.f};
  for (int j = 0; j < e.n_coll_act; ++j) w[e.act_map[j]] += e.act_scale[j] * a[j] / h;
  for (int i = 0; i < 4; ++i) u[i] = w[i];
}

// One thread per environment: choose the slot the step writes, store the step's actions,
// compute the collider's pose velocity.
__global__ void k_step_begin(const EnvDesc* __restrict__ envs, int env0, int n_env, const float* act_in, int a_max,
                             int record) {
  int ei = env0 + blockIdx.x * blockDim.x + threadIdx.x;
  if (ei >= env0 + n_env) return;
  const EnvDesc& e = envs[ei];
  EnvCtr* c = e.ctr;
  int live = c->live;
  c->next = record ? live + 1 : (live == 0 ? 1 : 0);
  const float* a = e.act_env ? e.act_env + (long long)c->t * e.A : act_in + (long long)ei * a_max;
  for (int j = 0; j < e.A; ++j) e.act[(long long)live * e.A + j] = a[j];
  pose_velocity(e, a, e.acc + ACC_U);
}

__device__ __forceinline__ float block_sum(float v, float* sh) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  const int w = threadIdx.x >> 5, l = threadIdx.x & 31;
  __syncthreads();
  if (l == 0) sh[w] = v;
  __syncthreads();
  float r = 0.f;
  const int nw = blockDim.x >> 5;
  for (int i = 0; i < nw; ++i) r += sh[i];
  return r;
}

// Reward statistics over the subsample (particles with caller id < n_sub) of a block.
// Two passes for the variance.  Returns (mean z, var z, mean v_x, n).
__device__ void subsample_stats(const EnvDesc& e, const float* b, float* sh, float* st) {
  const long long np = e.n_pad;
  const unsigned* meta = reinterpret_cast<const unsigned*>(b + kComp * np);
  const int ns = min(e.n_sub, e.n);
  float sz = 0.f, sv = 0.f;
  for (int i = threadIdx.x; i < e.n; i += blockDim.x) {
    if ((int)(meta[i] & kIdMask) < ns) {
      sz += b[2 * np + i];
      sv += b[3 * np + i];
    }
  }
  sz = block_sum(sz, sh);
  sv = block_sum(sv, sh);
  const float mz = sz / ns;
  float sq = 0.f;
  for (int i = threadIdx.x; i < e.n; i += blockDim.x) {
    if ((int)(meta[i] & kIdMask) < ns) {
      float d = b[2 * np + i] - mz;
      sq += d * d;
    }
  }
  sq = block_sum(sq, sh);
  st[0] = mz;
  st[1] = sq / ns;
  st[2] = sv / ns;
  st[3] = (float)ns;
}

__device__ __forceinline__ float rd_factor(float d, float thr) { return (d > thr) ? 1.0f : 2.0f; }

// One CTA per environment: reward of the finished step, end pose, counters.
__global__ void __launch_bounds__(256) k_reward_end(const EnvDesc* __restrict__ envs, int env0, float* reward_out,
                                                    int record) {
  __shared__ float sh[32];
  const int ei = env0 + blockIdx.x;
  const EnvDesc& e = envs[ei];
  EnvCtr* cp = e.ctr;
  const int live = cp->live, next = cp->next;
  const float* b = e.slots + (long long)next * e.block;
  float stats[4] = {0.f, 0.f, 0.f, 0.f};
  if (e.reward_kind == 1 || e.reward_kind == 3) subsample_stats(e, b, sh, stats);
  __syncthreads();
  if (threadIdx.x == 0) {
    const float h = e.S * e.dt;
    const int pl = pose_len(e);
    for (int i = 0; i < pl; ++i) e.pose[next * kPose + i] = e.pose[live * kPose + i] + h * e.acc[ACC_U + i];
    const float* qn = e.pose + next * kPose;  // body 0
    float r = 0.f;
    if (e.reward_kind == 1) {
      float d = stats[0] / e.rparam[0];
      r = rd_factor(d, 0.33f) / ((1.f + d) * (1.f + d)) - stats[1];
    } else if (e.reward_kind == 2) {
      float d = 0.f;
      for (int i = 0; i < 3; ++i) d += (qn[i] - e.rparam[i]) * (qn[i] - e.rparam[i]);
      r = rd_factor(d, 0.02f) / ((1.f + d) * (1.f + d));
    } else if (e.reward_kind == 3) {
      float aa = 0.f;
      for (int j = 0; j < e.A; ++j) {
        float a = e.act[(long long)live * e.A + j];
        aa += a * a;
      }
      r = stats[2] + e.rparam[1] * (stats[0] - e.rparam[0]) - e.rparam[2] * aa;
    }
    if (e.rew_env)
      e.rew_env[cp->t] = r;
    else if (reward_out)
      reward_out[ei] = r;
    cp->t += 1;
    cp->live = next;
    if (!record) cp->base = next;
  }
}

// ------------------------------------------------------------------ adjoint: G2P^T

template <int MAT, int BOX>
__global__ void __launch_bounds__(ScatterThreads<BOX>::value, BOX == kScBoxWarp ? 20 : 5)
    k_g2p_adj(const EnvDesc* __restrict__ envs, const WorkItem* __restrict__ items, int item_off, StateRef src,
              StateRef nxt, int use_perm, int k) {
  constexpr int NT = ScatterThreads<BOX>::value;
  __shared__ EnvDesc e;
  __shared__ EnvCtr c;
  __shared__ int sred[6];
  __shared__ ScatterShared<BOX> sh;
  WorkItem it;
  if (!scatter_part<NT>(items[item_off + blockIdx.x / (kBlock / NT)], it)) return;
  load_env(envs, it.env, e, c);
  const float* b = ref_block(e, c, src);
  const float* bn = ref_block(e, c, nxt);  // the substep's end state: holds v' and C'
  float* adj = c.par ? e.adj1 : e.adj0;
  const int sslot = step_slot(c, 1);
  const unsigned* perm = use_perm ? e.perm + (long long)sslot * e.n_pad : nullptr;
  const long long np = e.n_pad;
  const float G = (float)e.G;
  Mat m = env_mat(e);
  m.kind = MAT;  // compile-time material: the other laws' code is folded away
  const float Dinv = 4.0f * G * G, dt = e.dt, dx = e.dx;
  // reference = mean of v-bar + dt x-bar over the env's particles at this substep's end
  // (summed by P2G^T of the next substep, or by k_adj_ref for the step's last substep)
  const float inv_n = 1.0f / (float)e.n;
  const float* vs = e.acc + ACC_VSUM + 4 * (k & 1);
  const float vref[3] = {vs[0] * inv_n, vs[1] * inv_n, vs[2] * inv_n};
  if (it.start == 0 && threadIdx.x < 4) e.acc[ACC_VSUM + 4 * ((k + 1) & 1) + threadIdx.x] = 0.0f;
  int base[kPPT][3];
  bool valid[kPPT];
  int oob = 0;
#pragma unroll 1
  for (int p = 0; p < kPPT; ++p) {
    const int l = threadIdx.x + p * NT;
    valid[p] = l < it.count;
    sh.key[l] = 0xffffffffu;
    if (!valid[p]) continue;
    const int i = it.start + l;
    const int j = perm ? (int)perm[i] : i;
    float x[3], F[9];
#pragma unroll
    for (int a = 0; a < 3; ++a) x[a] = b[a * np + j];
#pragma unroll
    for (int a = 0; a < 9; ++a) F[a] = b[(15 + a) * np + j];
#pragma unroll
    for (int a = 0; a < 3; ++a) base[p][a] = cell_base(x[a], G, e.G, &oob);
    const int b0 = base[p][0], b1 = base[p][1], b2 = base[p][2];
    sh.key[l] = cell_pack(b0, b1, b2);
    float fx[3], w[3][3], dw[3][3];
#pragma unroll
    for (int a = 0; a < 3; ++a) {
      fx[a] = __fmul_rn(x[a], G) - (float)base[p][a];
      bspline(fx[a], w[a], dw[a]);
#pragma unroll
      for (int o = 0; o < 3; ++o) dw[a][o] *= G;
    }
    // v' and C' as the forward G2P stored them in the substep's end state
    float Cn[9];
#pragma unroll
    for (int a = 0; a < 9; ++a) Cn[a] = bn[(6 + a) * np + i];
    const float4 vc = __ldg(e.grid_v + ((long long)(b2 + 1) * e.G + (b1 + 1)) * e.G + b0 + 1);
    // trial H_t = H + dt (C' + C' H)   (F here holds H = F - I)
    float CH[9], Ft[9];
    matmul3(Cn, F, CH);
#pragma unroll
    for (int a = 0; a < 9; ++a) Ft[a] = F[a] + dt * (Cn[a] + CH[a]);
    // incoming adjoint of the end state
    float xb[3], vb[3], Cb[9], Fob[9];
#pragma unroll
    for (int a = 0; a < 3; ++a) {
      xb[a] = adj[a * np + i];
      vb[a] = adj[(3 + a) * np + i];
    }
#pragma unroll
    for (int a = 0; a < 9; ++a) {
      Cb[a] = adj[(6 + a) * np + i];
      Fob[a] = adj[(15 + a) * np + i];
    }
    float Ftb[9];
    project_vjp(m, Ft, Fob, Ftb);
    // F_t = (I + dt C') F:  Cb += dt Ftb F^T = dt (Ftb + Ftb H^T);  Fb_partial = Ftb + dt C'^T Ftb
#pragma unroll
    for (int a = 0; a < 3; ++a)
#pragma unroll
      for (int bb = 0; bb < 3; ++bb) {
        Cb[3 * a + bb] += dt * (Ftb[3 * a + bb] + Ftb[3 * a] * F[3 * bb] + Ftb[3 * a + 1] * F[3 * bb + 1] +
                                Ftb[3 * a + 2] * F[3 * bb + 2]);
        adj[(15 + 3 * a + bb) * np + i] =
            Ftb[3 * a + bb] + dt * (Cn[a] * Ftb[bb] + Cn[3 + a] * Ftb[3 + bb] + Cn[6 + a] * Ftb[6 + bb]);
      }
    // x' = x + dt v';  A' = D^-1 C-bar
    const float vnb[3] = {vb[0] + dt * xb[0], vb[1] + dt * xb[1], vb[2] + dt * xb[2]};
    float Ab[9];
#pragma unroll
    for (int a = 0; a < 9; ++a) Ab[a] = Dinv * Cb[a];
    // scatter record: the grid receives sum w (v-bar' - V_ref + A' r); V_ref m_i / m_p is
    // restored in the grid adjoint
    {
      const float q[3] = {vnb[0] - vref[0], vnb[1] - vref[1], vnb[2] - vref[2]};
      const float g[3] = {fx[0] * dx, fx[1] * dx, fx[2] * dx};
      write_record<NT * kPPT>(sh.rec + l, q, g, w[0], w[1], w[2], Ab);
    }
    // gather: x-bar += sum_i (g_i . (v-bar' + A' r_i)) grad w_i - A'^T sum_i w_i g_i with
    // g_i = v_i - v_c (the stencil-uniform part of v_i adds nothing: sum grad w = 0 and
    // sum r grad w^T = I cancel it against the w C-bar^T term)
    float xbp[3] = {xb[0], xb[1], xb[2]};
    float swg[3] = {0.f, 0.f, 0.f};
#pragma unroll
    for (int oc = 0; oc < 3; ++oc) {
      // the layer's nine nodes are loaded together, so that their latencies overlap (loading
      // row by row ran 4% slower; loading by layers with 128 registers a thread, 5% slower)
      float4 gl[3][3];
#pragma unroll
      for (int ob = 0; ob < 3; ++ob)
#pragma unroll
        for (int oa = 0; oa < 3; ++oa)
          gl[ob][oa] = __ldg(e.grid_v + ((long long)(b2 + oc) * e.G + (b1 + ob)) * e.G + b0 + oa);
#pragma unroll
      for (int ob = 0; ob < 3; ++ob) {
        const float wyz = w[1][ob] * w[2][oc], dwy_wz = dw[1][ob] * w[2][oc], wy_dwz = w[1][ob] * dw[2][oc];
        const float ry = ((float)ob - fx[1]) * dx, rz = ((float)oc - fx[2]) * dx;
        const float q0 = vnb[0] + Ab[1] * ry + Ab[2] * rz;
        const float q1 = vnb[1] + Ab[4] * ry + Ab[5] * rz;
        const float q2 = vnb[2] + Ab[7] * ry + Ab[8] * rz;
        // the row's sums over x first; its y and z factors are applied once
        float sd = 0.f, sw = 0.f, gw0 = 0.f, gw1 = 0.f, gw2 = 0.f;
#pragma unroll
        for (int oa = 0; oa < 3; ++oa) {
          const float4 gv = gl[ob][oa];
          const float g0 = gv.x - vc.x, g1 = gv.y - vc.y, g2 = gv.z - vc.z;
          const float rx = ((float)oa - fx[0]) * dx;
          const float sdw = g0 * (q0 + Ab[0] * rx) + g1 * (q1 + Ab[3] * rx) + g2 * (q2 + Ab[6] * rx);
          sd += sdw * dw[0][oa];
          sw += sdw * w[0][oa];
          gw0 += w[0][oa] * g0;
          gw1 += w[0][oa] * g1;
          gw2 += w[0][oa] * g2;
        }
        xbp[0] += sd * wyz;
        xbp[1] += sw * dwy_wz;
        xbp[2] += sw * wy_dwz;
        swg[0] += gw0 * wyz;
        swg[1] += gw1 * wyz;
        swg[2] += gw2 * wyz;
      }
    }
#pragma unroll
    for (int a = 0; a < 3; ++a) adj[a * np + i] = xbp[a] - (Ab[a] * swg[0] + Ab[3 + a] * swg[1] + Ab[6 + a] * swg[2]);
  }
  (void)oob;
  const Box bx = make_box(base, valid, sred);
  scatter_groups<false, BOX>(sh, e, it.env, it.count, valid, base, sred, bx, 0.0f, e.grid_vb, nullptr, nullptr);
}

// ------------------------------------------------------------------ adjoint: grid^T

// Reverse of node_forward for the velocity adjoint vob (linear in vob), given its trace t.
__device__ __forceinline__ void node_reverse(const EnvDesc& e, int ix, int iy, int iz, float4 mp, const float* q,
                                             const float* u, const NodeFwd& t, float4 vob, float4& mpb, float* qb,
                                             float* ub) {
  float v3b[3] = {(t.zero & 1u) ? 0.f : vob.x, (t.zero & 2u) ? 0.f : vob.y, (t.zero & 4u) ? 0.f : vob.z};
  float v2b[3];
  if (t.ground) {
    if (e.ground_mu > 0.0f) {
      if (t.gL > 0.0f && t.gf > 0.0f) {
        const float dot = v3b[0] * t.v2[0] + v3b[1] * t.v2[1];
        const float iL3 = 1.0f / (t.gL * t.gL * t.gL);
        v2b[0] = t.gf * v3b[0] - dot * e.ground_mu * t.v2[2] * t.v2[0] * iL3;
        v2b[1] = t.gf * v3b[1] - dot * e.ground_mu * t.v2[2] * t.v2[1] * iL3;
        v2b[2] = dot * e.ground_mu / t.gL;
      } else {
        v2b[0] = v2b[1] = v2b[2] = 0.0f;
      }
    } else {
      v2b[0] = v3b[0];
      v2b[1] = v3b[1];
      v2b[2] = 0.0f;
    }
  } else {
    v2b[0] = v3b[0];
    v2b[1] = v3b[1];
    v2b[2] = v3b[2];
  }
  float v1b[3];
  if (e.coll_kind != COLL_NONE) {
    const float sc = t.sc;
    float scb = 0.0f;
#pragma unroll
    for (int i = 0; i < 3; ++i) {
      v1b[i] = (1.0f - sc) * v2b[i];
      scb += v2b[i] * t.dl[i];
    }
    float vr2b[3] = {sc * v2b[0], sc * v2b[1], sc * v2b[2]};
    float vbb[3] = {vr2b[0], vr2b[1], vr2b[2]};
    float vrb[3] = {0.f, 0.f, 0.f}, nb[3] = {0.f, 0.f, 0.f};
    if (t.branch == 0) {
#pragma unroll
      for (int i = 0; i < 3; ++i) vrb[i] = vr2b[i];
    } else if (t.branch == 1) {
      const float dot = vr2b[0] * t.vt[0] + vr2b[1] * t.vt[1] + vr2b[2] * t.vt[2];
      const float iL = 1.0f / t.L;
      const float c3 = dot * e.coll_mu * t.vn * iL * iL * iL;
      float vtb[3];
#pragma unroll
      for (int i = 0; i < 3; ++i) vtb[i] = t.f * vr2b[i] - c3 * t.vt[i];
      float vnb = dot * e.coll_mu * iL;
#pragma unroll
      for (int i = 0; i < 3; ++i) {
        vrb[i] += vtb[i];
        nb[i] -= t.vn * vtb[i];
      }
      vnb -= vtb[0] * t.ct.n[0] + vtb[1] * t.ct.n[1] + vtb[2] * t.ct.n[2];
#pragma unroll
      for (int i = 0; i < 3; ++i) {
        vrb[i] += vnb * t.ct.n[i];
        nb[i] += vnb * t.vr[i];
      }
    }
#pragma unroll
    for (int i = 0; i < 3; ++i) {
      v1b[i] += vrb[i];
      vbb[i] -= vrb[i];
    }
    const float db = t.ct.d > 0.0f ? scb * (-e.alpha * sc) : 0.0f;
    const float* H = t.ct.H;  // xx xy xz yy yz zz
    const float Hn0 = H[0] * nb[0] + H[1] * nb[1] + H[2] * nb[2];
    const float Hn1 = H[1] * nb[0] + H[3] * nb[1] + H[4] * nb[2];
    const float Hn2 = H[2] * nb[0] + H[4] * nb[1] + H[5] * nb[2];
    qb[0] += -t.ct.n[0] * db - Hn0 - u[3] * vbb[1];
    qb[1] += -t.ct.n[1] * db - Hn1 + u[3] * vbb[0];
    qb[2] += -t.ct.n[2] * db - Hn2;
    qb[3] += t.ct.dd_dth * db + t.ct.dn_dth[0] * nb[0] + t.ct.dn_dth[1] * nb[1] + t.ct.dn_dth[2] * nb[2];
    const float rx = ix * e.dx - q[0], ry = iy * e.dx - q[1];
    ub[0] += vbb[0];
    ub[1] += vbb[1];
    ub[2] += vbb[2];
    ub[3] += -ry * vbb[0] + rx * vbb[1];
  } else {
    v1b[0] = v2b[0];
    v1b[1] = v2b[1];
    v1b[2] = v2b[2];
  }
  const float inv_m = 1.0f / mp.x;
  mpb.x = -(v1b[0] * t.v0[0] + v1b[1] * t.v0[1] + v1b[2] * t.v0[2]) * inv_m;
  mpb.y = v1b[0] * inv_m;
  mpb.z = v1b[1] * inv_m;
  mpb.w = v1b[2] * inv_m;
}

__global__ void __launch_bounds__(256) k_grid_adj(const EnvDesc* __restrict__ envs, const uint2* __restrict__ active,
                                                  const int* __restrict__ active_n, int k) {
  const int lane = threadIdx.x & 31;
  const int warp = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const int nwarps = (gridDim.x * blockDim.x) >> 5;
  const int n = *active_n;
  for (int w = warp; w < n; w += nwarps) {
    const uint2 at = active[w];
    const EnvDesc& e = envs[at.x];
    const EnvCtr c = *e.ctr;
    float q0[4], u0[4];
    const float* ps = step_pose(e, c, 1, k, q0, u0);
    float st0, ct0;
    sincosf(q0[3], &st0, &ct0);
    const float kdt = (float)k * e.dt;
    const int TG = e.G >> 2;
    const int tz = at.y / (TG * TG), ty = (at.y / TG) % TG, tx = at.y % TG;
    float qb[4] = {0.f, 0.f, 0.f, 0.f}, ub[4] = {0.f, 0.f, 0.f, 0.f};
    const float inv_n = 1.0f / (float)e.n;
    const float* vs = e.acc + ACC_VSUM + 4 * (k & 1);
    const float vref[3] = {vs[0] * inv_n, vs[1] * inv_n, vs[2] * inv_n};
    const float inv_pm = 1.0f / e.p_mass;
#pragma unroll 1
    for (int h = 0; h < 2; ++h) {
      const int l = lane + 32 * h;
      const int ix = tx * 4 + (l & 3), iy = ty * 4 + ((l >> 2) & 3), iz = tz * 4 + (l >> 4);
      const long long id = ((long long)iz * e.G + iy) * e.G + ix;
      const float4 mp = e.grid_mp[id];
      float4 mpb = make_float4(0.f, 0.f, 0.f, 0.f);
      // pose adjoints of this node (capsule union: of capsule `which`)
      float qn[4] = {0.f, 0.f, 0.f, 0.f}, un[4] = {0.f, 0.f, 0.f, 0.f};
      int which = -1;
      if (mp.x > 0.0f) {
        // grid_vb holds sum w (v-bar' - V_ref); the full adjoint is that + V_ref m / m_p
        const float4 vd = e.grid_vb[id];
        NodeFwd t;
        float q[4] = {q0[0], q0[1], q0[2], q0[3]}, u[4] = {u0[0], u0[1], u0[2], u0[3]};
        node_forward<true>(e, ix, iy, iz, mp, q, u, ps, kdt, st0, ct0, t);
        const bool ident = t.zero == 0u && !t.ground && (e.coll_kind == COLL_NONE || t.sc == 0.0f);
        if (ident) {
          // the node update is the identity map on velocities here: p-bar = v-bar/m exactly,
          // with the V_ref part a single FP32 constant (it cancels exactly in P2G^T)
          const float inv_m = 1.0f / mp.x;
          const float r0 = vref[0] * inv_pm, r1 = vref[1] * inv_pm, r2 = vref[2] * inv_pm;
          mpb.y = vd.x * inv_m + r0;
          mpb.z = vd.y * inv_m + r1;
          mpb.w = vd.z * inv_m + r2;
          mpb.x = -((vd.x * t.v0[0] + vd.y * t.v0[1] + vd.z * t.v0[2]) * inv_m +
                    (r0 * t.v0[0] + r1 * t.v0[1] + r2 * t.v0[2]));
        } else {
          const float sc = mp.x * inv_pm;
          const float4 vob = make_float4(vd.x + vref[0] * sc, vd.y + vref[1] * sc, vd.z + vref[2] * sc, 0.f);
          node_reverse(e, ix, iy, iz, mp, q, u, t, vob, mpb, qn, un);
          which = t.which;
        }
      }
      e.grid_mpb[id] = mpb;
      e.grid_mp[id] = make_float4(0.f, 0.f, 0.f, 0.f);
      e.grid_vb[id] = make_float4(0.f, 0.f, 0.f, 0.f);
      if (e.coll_kind == COLL_CAPSULES) {
        // the nodes of a warp may touch different capsules: one warp sum per capsule present
        unsigned present = __reduce_or_sync(0xffffffffu, which >= 0 ? 1u << which : 0u);
        while (present) {
          const int j = __ffs(present) - 1;
          present &= present - 1u;
          const bool mine = which == j;
#pragma unroll
          for (int i = 0; i < 4; ++i) {
            float a = mine ? qn[i] : 0.0f, b2 = mine ? un[i] : 0.0f;
#pragma unroll
            for (int o = 16; o > 0; o >>= 1) {
              a += __shfl_xor_sync(0xffffffffu, a, o);
              b2 += __shfl_xor_sync(0xffffffffu, b2, o);
            }
            if (lane == 0) {
              if (a != 0.0f) {
                atomicAdd(e.acc + ACC_QKB + 4 * j + i, a);
                atomicAdd(e.acc + ACC_KQKB + 4 * j + i, kdt * a);
              }
              if (b2 != 0.0f) atomicAdd(e.acc + ACC_UB + 4 * j + i, b2);
            }
          }
        }
      } else {
#pragma unroll
        for (int i = 0; i < 4; ++i) {
          qb[i] += qn[i];
          ub[i] += un[i];
        }
      }
    }
    if (e.coll_kind != COLL_NONE && e.coll_kind != COLL_CAPSULES) {
#pragma unroll
      for (int i = 0; i < 4; ++i) {
        float a = qb[i], b2 = ub[i];
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) {
          a += __shfl_xor_sync(0xffffffffu, a, o);
          b2 += __shfl_xor_sync(0xffffffffu, b2, o);
        }
        qb[i] = a;
        ub[i] = b2;
      }
      if (lane == 0) {
#pragma unroll
        for (int i = 0; i < 4; ++i) {
          if (qb[i] != 0.0f) {
            atomicAdd(e.acc + ACC_QKB + i, qb[i]);
            atomicAdd(e.acc + ACC_KQKB + i, kdt * qb[i]);
          }
          if (ub[i] != 0.0f) atomicAdd(e.acc + ACC_UB + i, ub[i]);
        }
      }
    }
    if (lane == 0) e.tile[at.y] = 0u;
  }
}

// ------------------------------------------------------------------ adjoint: P2G^T

template <int MAT>
__global__ void __launch_bounds__(kBlock, 6) k_p2g_adj(const EnvDesc* __restrict__ envs,
                                                       const WorkItem* __restrict__ items, int item_off, StateRef src,
                                                       int use_perm, int k) {
  __shared__ float vsum_s[3];
  __shared__ EnvDesc e;
  __shared__ EnvCtr c;
  const WorkItem it = items[item_off + blockIdx.x];
  load_env(envs, it.env, e, c);
  const float* b = ref_block(e, c, src);
  float* adj = c.par ? e.adj1 : e.adj0;
  float* adj_out = use_perm ? (c.par ? e.adj0 : e.adj1) : adj;
  const int sslot = step_slot(c, 1);
  const unsigned* perm = use_perm ? e.perm + (long long)sslot * e.n_pad : nullptr;
  const long long np = e.n_pad;
  const float G = (float)e.G;
  Mat m = env_mat(e);
  m.kind = MAT;  // compile-time material: the other laws' code is folded away
  const float Dinv = 4.0f * G * G, dx = e.dx, pm = e.p_mass;
  const float stress_k = -e.dt * e.p_vol * Dinv;
  if (threadIdx.x < 3) vsum_s[threadIdx.x] = 0.0f;
  __syncthreads();
  float vsum[3] = {0.f, 0.f, 0.f};
#pragma unroll 1
  for (int p = 0; p < kPPT; ++p) {
    const int i = it.start + threadIdx.x + p * kBlock;
    if (i >= it.start + it.count) continue;
    const int j = perm ? (int)perm[i] : i;
    float s[kComp];
    load_state(b, np, j, s);
    const unsigned meta = reinterpret_cast<const unsigned*>(b + kComp * np)[j];
    const float a_g = MAT == MAT_MUSCLE ? group_act(e, sslot, meta) : 0.0f;
    int base[3], oob = 0;
    float fx[3], w[3][3], dwv[3][3];
#pragma unroll
    for (int a = 0; a < 3; ++a) {
      base[a] = cell_base(s[a], G, e.G, &oob);
      fx[a] = __fmul_rn(s[a], G) - (float)base[a];
      bspline(fx[a], w[a], dwv[a]);
    }
    float tau[9], A[9];
    kirchhoff(m, s + 15, s + 6, a_g, tau);
#pragma unroll
    for (int q = 0; q < 9; ++q) A[q] = pm * s[6 + q] + stress_k * tau[q];
    // The stencil-centre node's (m-bar, p-bar) adds nothing to A-bar and x-bar (sum w r = 0,
    // sum grad w = 0, sum r grad w^T = I); subtracting it keeps the FP32 sums from cancelling.
    const float4 gc =
        __ldg(e.grid_mpb + ((long long)(base[2] + 1) * e.G + (base[1] + 1)) * e.G + base[0] + 1);
    // Per node i (p-bar_i relative to the centre): u = w p-bar;  A-bar += u r^T;  S += u;
    // x-bar += (m-bar_i m_p + p-bar_i . (m_p v + A r)) grad w.  After the stencil:
    // v-bar = m_p (S + p-bar_c sum w) and x-bar -= A^T S.  The weights are separable: each
    // row of three nodes is summed over x first (with w_x, w_x r_x, dw_x) and the row's y and
    // z factors are applied once.
    float Ab[9], S[3] = {0.f, 0.f, 0.f}, xbn[3] = {0.f, 0.f, 0.f};
#pragma unroll
    for (int q = 0; q < 9; ++q) Ab[q] = 0.f;
    float rx[3], gwx[3], wxr[3];
#pragma unroll
    for (int o = 0; o < 3; ++o) {
      rx[o] = ((float)o - fx[0]) * dx;
      gwx[o] = dwv[0][o] * G;
      wxr[o] = w[0][o] * rx[o];
    }
    const float sw = (w[0][0] + w[0][1] + w[0][2]) * (w[1][0] + w[1][1] + w[1][2]) * (w[2][0] + w[2][1] + w[2][2]);
    const float mv0 = pm * s[3], mv1 = pm * s[4], mv2 = pm * s[5];
#pragma unroll 1
    for (int cz = 0; cz < 3; ++cz) {
      const float wz = cz == 0 ? w[2][0] : (cz == 1 ? w[2][1] : w[2][2]);
      const float dwz = (cz == 0 ? dwv[2][0] : (cz == 1 ? dwv[2][1] : dwv[2][2])) * G;
      const float rz = ((float)cz - fx[2]) * dx;
#pragma unroll
      for (int cy = 0; cy < 3; ++cy) {
        const float wyz = w[1][cy] * wz, dwy_wz = dwv[1][cy] * G * wz, wy_dwz = w[1][cy] * dwz;
        const float ry = ((float)cy - fx[1]) * dx;
        const float q0 = mv0 + A[1] * ry + A[2] * rz;
        const float q1 = mv1 + A[4] * ry + A[5] * rz;
        const float q2 = mv2 + A[7] * ry + A[8] * rz;
        const float4* row = e.grid_mpb + ((long long)(base[2] + cz) * e.G + (base[1] + cy)) * e.G + base[0];
        float r0[3] = {0.f, 0.f, 0.f}, r1[3] = {0.f, 0.f, 0.f};  // sum_a w_x p-bar, sum_a w_x r_x p-bar
        float k0 = 0.f, k1 = 0.f;                                 // sum_a dw_x coef, sum_a w_x coef
#pragma unroll
        for (int cx = 0; cx < 3; ++cx) {
          const float4 gb = __ldg(row + cx);
          const float p0 = gb.y - gc.y, p1 = gb.z - gc.z, p2 = gb.w - gc.w;
          r0[0] += w[0][cx] * p0;
          r0[1] += w[0][cx] * p1;
          r0[2] += w[0][cx] * p2;
          r1[0] += wxr[cx] * p0;
          r1[1] += wxr[cx] * p1;
          r1[2] += wxr[cx] * p2;
          const float coef = (gb.x - gc.x) * pm + p0 * q0 + p1 * q1 + p2 * q2 +
                             rx[cx] * (p0 * A[0] + p1 * A[3] + p2 * A[6]);
          k0 += gwx[cx] * coef;
          k1 += w[0][cx] * coef;
        }
        const float wyr = wyz * ry, wzr = wyz * rz;
#pragma unroll
        for (int q = 0; q < 3; ++q) {
          S[q] += wyz * r0[q];
          Ab[3 * q] += wyz * r1[q];
          Ab[3 * q + 1] += wyr * r0[q];
          Ab[3 * q + 2] += wzr * r0[q];
        }
        xbn[0] += wyz * k0;
        xbn[1] += dwy_wz * k1;
        xbn[2] += wy_dwz * k1;
      }
    }
    const float vbn[3] = {pm * (S[0] + gc.y * sw), pm * (S[1] + gc.z * sw), pm * (S[2] + gc.w * sw)};
#pragma unroll
    for (int a = 0; a < 3; ++a) xbn[a] -= A[a] * S[0] + A[3 + a] * S[1] + A[6 + a] * S[2];
    float Cbn[9], taub[9], Fbn[9];
#pragma unroll
    for (int q = 0; q < 9; ++q) {
      Cbn[q] = pm * Ab[q];
      taub[q] = stress_k * Ab[q];
      Fbn[q] = adj[(15 + q) * np + i];
    }
    // C and H again (cached): not holding them through the stencil loop saves registers
    float CH[18];
#pragma unroll
    for (int q = 0; q < 18; ++q) CH[q] = b[(6 + q) * np + j];
    float agb = 0.0f;
    kirchhoff_vjp(m, CH + 9, CH, a_g, taub, Fbn, Cbn, &agb);
    const int o = perm ? j : i;
#pragma unroll
    for (int a = 0; a < 3; ++a) {
      const float xp = adj[a * np + i];
      adj_out[a * np + o] = xp + xbn[a];
      adj_out[(3 + a) * np + o] = vbn[a];
      vsum[a] += vbn[a] + e.dt * (xp + xbn[a]);
    }
#pragma unroll
    for (int q = 0; q < 9; ++q) {
      adj_out[(6 + q) * np + o] = Cbn[q];
      adj_out[(15 + q) * np + o] = Fbn[q];
    }
    if (MAT == MAT_MUSCLE) {
      const int g = (int)(meta >> 20) - 1;
      if (g >= 0 && g < e.n_groups) atomicAdd(e.acc + ACC_ACT + e.n_coll_act + g, agb);
    }
  }
  // per-env sum of the produced adjoint (v-bar + dt x-bar): the reference of substep k-1
#pragma unroll
  for (int a = 0; a < 3; ++a) {
    float v = vsum[a];
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    if ((threadIdx.x & 31) == 0) atomicAdd(&vsum_s[a], v);
  }
  __syncthreads();
  if (threadIdx.x < 3) atomicAdd(e.acc + ACC_VSUM + 4 * ((k + 1) & 1) + threadIdx.x, vsum_s[threadIdx.x]);
}

// ------------------------------------------------------------------ reverse-step bookkeeping

// Start of a reverse pass over T steps: adjoint parity 0, pose adjoint 0, step index T.
__global__ void k_bwd_init(const EnvDesc* __restrict__ envs, int env0, int n_env, int T) {
  int ei = env0 + blockIdx.x * blockDim.x + threadIdx.x;
  if (ei >= env0 + n_env) return;
  const EnvDesc& e = envs[ei];
  e.ctr->par = 0;
  e.ctr->rev = T;
  for (int i = 0; i < kPose; ++i) e.acc[ACC_QB + i] = 0.f;
}

// Next step of the reverse pass: t = rev - 1; pose velocity of step t; zero accumulators.
__global__ void k_rev_begin(const EnvDesc* __restrict__ envs, int env0, int n_env) {
  int ei = env0 + blockIdx.x * blockDim.x + threadIdx.x;
  if (ei >= env0 + n_env) return;
  const EnvDesc& e = envs[ei];
  EnvCtr* c = e.ctr;
  const int t = c->rev - 1;
  c->rev = t;
  const int slot = c->base + t;
  pose_velocity(e, e.act + (long long)slot * e.A, e.acc + ACC_U);
  for (int i = 0; i < kPose; ++i) {
    e.acc[ACC_QKB + i] = 0.f;
    e.acc[ACC_KQKB + i] = 0.f;
    e.acc[ACC_UB + i] = 0.f;
  }
  for (int j = 0; j < e.A; ++j) e.acc[ACC_ACT + j] = 0.f;
}

// One CTA per env: add rbar_t * d r_t / d(end state, end pose, action).
__global__ void __launch_bounds__(256) k_reward_adj(const EnvDesc* __restrict__ envs, int env0, const float* rbar,
                                                    int n_tot) {
  __shared__ float sh[32];
  const int ei = env0 + blockIdx.x;
  const EnvDesc& e = envs[ei];
  const EnvCtr c = *e.ctr;
  const float rb = e.rbar_env ? e.rbar_env[c.rev] : (rbar ? rbar[(long long)c.rev * n_tot + ei] : 0.0f);
  if (rb == 0.0f || e.reward_kind == 0) return;
  const int slot = c.base + c.rev;
  const float* b = e.slots + (long long)(slot + 1) * e.block;
  float* adj = c.par ? e.adj1 : e.adj0;
  const long long np = e.n_pad;
  const unsigned* meta = reinterpret_cast<const unsigned*>(b + kComp * np);
  const int ns = min(e.n_sub, e.n);
  if (e.reward_kind == 1) {
    float st[4];
    subsample_stats(e, b, sh, st);
    const float d = st[0] / e.rparam[0];
    const float dRd = -2.0f * rd_factor(d, 0.33f) / ((1.f + d) * (1.f + d) * (1.f + d));
    for (int i = threadIdx.x; i < e.n; i += blockDim.x)
      if ((int)(meta[i] & kIdMask) < ns)
        adj[2 * np + i] += rb * (dRd / (e.rparam[0] * ns) - 2.0f * (b[2 * np + i] - st[0]) / ns);
  } else if (e.reward_kind == 2) {
    if (threadIdx.x == 0) {
      const float* q = e.pose + (slot + 1) * kPose;
      float d = 0.f;
      for (int i = 0; i < 3; ++i) d += (q[i] - e.rparam[i]) * (q[i] - e.rparam[i]);
      const float dRd = -2.0f * rd_factor(d, 0.02f) / ((1.f + d) * (1.f + d) * (1.f + d));
      for (int i = 0; i < 3; ++i) e.acc[ACC_QB + i] += rb * dRd * 2.0f * (q[i] - e.rparam[i]);
    }
  } else if (e.reward_kind == 3) {
    for (int i = threadIdx.x; i < e.n; i += blockDim.x)
      if ((int)(meta[i] & kIdMask) < ns) {
        adj[3 * np + i] += rb / ns;
        adj[2 * np + i] += rb * e.rparam[1] / ns;
      }
    if (threadIdx.x == 0)
      for (int j = 0; j < e.A; ++j) e.acc[ACC_ACT + j] += rb * (-2.0f * e.rparam[2] * e.act[(long long)slot * e.A + j]);
  }
}

// One CTA per env: sum over the env's particles of the adjoint v-bar + dt x-bar of the step's
// end state, the reference of the step's last substep (any value is exact; the mean of the
// current adjoint keeps the shifted adjoint small).
__global__ void __launch_bounds__(256) k_adj_ref(const EnvDesc* __restrict__ envs, int env0) {
  __shared__ float sh[32];
  const int ei = env0 + blockIdx.x;
  const EnvDesc& e = envs[ei];
  const EnvCtr c = *e.ctr;
  const float* adj = c.par ? e.adj1 : e.adj0;
  const long long np = e.n_pad;
  float s0 = 0.f, s1 = 0.f, s2 = 0.f;
  for (int i = threadIdx.x; i < e.n; i += blockDim.x) {
    s0 += adj[3 * np + i] + e.dt * adj[i];
    s1 += adj[4 * np + i] + e.dt * adj[np + i];
    s2 += adj[5 * np + i] + e.dt * adj[2 * np + i];
  }
  s0 = block_sum(s0, sh);
  s1 = block_sum(s1, sh);
  s2 = block_sum(s2, sh);
  if (threadIdx.x == 0) {
    float* vs = e.acc + ACC_VSUM + 4 * ((e.S - 1) & 1);
    vs[0] = s0;
    vs[1] = s1;
    vs[2] = s2;
  }
}

__global__ void k_rev_end(const EnvDesc* __restrict__ envs, int env0, int n_env, float* act_grad, int n_tot,
                          int a_max) {
  int ei = env0 + blockIdx.x * blockDim.x + threadIdx.x;
  if (ei >= env0 + n_env) return;
  const EnvDesc& e = envs[ei];
  EnvCtr* c = e.ctr;
  const float h = e.S * e.dt;
  // q_k = q_t + k dt u for the step's substeps and q_{t+1} = q_t + h u: the adjoint of u is
  // h qb_{t+1} + sum_k k dt qb_k + (through the body velocity) ub, and qb_t = qb_{t+1} + sum_k qb_k
  const int pl = pose_len(e);
  float* ub = e.acc + ACC_UB;
  for (int i = 0; i < pl; ++i) {
    ub[i] += h * e.acc[ACC_QB + i] + e.acc[ACC_KQKB + i];
    e.acc[ACC_QB + i] += e.acc[ACC_QKB + i];
  }
  float* out;
  int width;
  if (e.agrad_env) {
    out = e.agrad_env + (long long)c->rev * e.A;
    width = e.A;
  } else {
    out = act_grad + ((long long)c->rev * n_tot + ei) * a_max;
    width = a_max;
  }
  for (int j = 0; j < width; ++j) {
    float g = 0.f;
    if (j < e.A) {
      g = e.acc[ACC_ACT + j];
      if (j < e.n_coll_act)
        g += (e.coll_kind == COLL_CAPSULES ? ub[j] * e.act_scale[j & 3] : ub[e.act_map[j]] * e.act_scale[j]) / h;
    }
    out[j] = g;
  }
  c->par ^= 1;
}

// ------------------------------------------------------------------ state I/O

// Caller order (particle-major AoS) -> slot 0, meta = id | (group+1) << 20.
__global__ void k_set_state(const EnvDesc* __restrict__ envs, const WorkItem* __restrict__ items, int item_off,
                            const float* x, const float* v, const float* C, const float* F, const int* group) {
  const WorkItem it = items[item_off + blockIdx.x];
  const EnvDesc& e = envs[it.env];
  float* b = e.slots;
  const long long np = e.n_pad;
  for (int p = threadIdx.x; p < it.count; p += blockDim.x) {
    const int i = it.start + p;
    const long long g = e.poff + i;
#pragma unroll
    for (int a = 0; a < 3; ++a) {
      b[a * np + i] = x[g * 3 + a];
      b[(3 + a) * np + i] = v[g * 3 + a];
    }
#pragma unroll
    for (int a = 0; a < 9; ++a) {
      b[(6 + a) * np + i] = C[g * 9 + a];
      b[(15 + a) * np + i] = F[g * 9 + a] - ((a % 4 == 0) ? 1.0f : 0.0f);  // stored as H = F - I
    }
    int gr = group ? group[g] : -1;
    if (gr < -1 || gr > 4094) gr = -1;
    reinterpret_cast<unsigned*>(b + kComp * np)[i] = (unsigned)i | ((unsigned)(gr + 1) << 20);
  }
}

// block -> caller order by meta id.
__global__ void k_get_state(const EnvDesc* __restrict__ envs, const WorkItem* __restrict__ items, int item_off,
                            StateRef src, float* x, float* v, float* C, float* F) {
  __shared__ EnvDesc e;
  __shared__ EnvCtr c;
  const WorkItem it = items[item_off + blockIdx.x];
  load_env(envs, it.env, e, c);
  const float* b = ref_block(e, c, src);
  const long long np = e.n_pad;
  for (int p = threadIdx.x; p < it.count; p += blockDim.x) {
    const int i = it.start + p;
    const long long g = e.poff + (reinterpret_cast<const unsigned*>(b + kComp * np)[i] & kIdMask);
#pragma unroll
    for (int a = 0; a < 3; ++a) {
      if (x) x[g * 3 + a] = b[a * np + i];
      if (v) v[g * 3 + a] = b[(3 + a) * np + i];
    }
#pragma unroll
    for (int a = 0; a < 9; ++a) {
      if (C) C[g * 9 + a] = b[(6 + a) * np + i];
      if (F) F[g * 9 + a] = b[(15 + a) * np + i] + ((a % 4 == 0) ? 1.0f : 0.0f);
    }
  }
}

// Caller-order adjoint of the live state -> adj[par] in the live block's order.
__global__ void k_adj_in(const EnvDesc* __restrict__ envs, const WorkItem* __restrict__ items, int item_off,
                         const float* xb, const float* vb, const float* Cb, const float* Fb) {
  __shared__ EnvDesc e;
  __shared__ EnvCtr c;
  const WorkItem it = items[item_off + blockIdx.x];
  load_env(envs, it.env, e, c);
  const float* b = e.slots + (long long)c.live * e.block;
  float* adj = c.par ? e.adj1 : e.adj0;
  const long long np = e.n_pad;
  for (int p = threadIdx.x; p < it.count; p += blockDim.x) {
    const int i = it.start + p;
    const long long g = e.poff + (reinterpret_cast<const unsigned*>(b + kComp * np)[i] & kIdMask);
#pragma unroll
    for (int a = 0; a < 3; ++a) {
      adj[a * np + i] = xb ? xb[g * 3 + a] : 0.f;
      adj[(3 + a) * np + i] = vb ? vb[g * 3 + a] : 0.f;
    }
#pragma unroll
    for (int a = 0; a < 9; ++a) {
      adj[(6 + a) * np + i] = Cb ? Cb[g * 9 + a] : 0.f;
      adj[(15 + a) * np + i] = Fb ? Fb[g * 9 + a] : 0.f;
    }
  }
}

// adj[par] (order of block src) -> caller order.
__global__ void k_adj_out(const EnvDesc* __restrict__ envs, const WorkItem* __restrict__ items, int item_off,
                          StateRef src, float* xb, float* vb, float* Cb, float* Fb) {
  __shared__ EnvDesc e;
  __shared__ EnvCtr c;
  const WorkItem it = items[item_off + blockIdx.x];
  load_env(envs, it.env, e, c);
  const float* b = ref_block(e, c, src);
  const float* adj = c.par ? e.adj1 : e.adj0;
  const long long np = e.n_pad;
  for (int p = threadIdx.x; p < it.count; p += blockDim.x) {
    const int i = it.start + p;
    const long long g = e.poff + (reinterpret_cast<const unsigned*>(b + kComp * np)[i] & kIdMask);
#pragma unroll
    for (int a = 0; a < 3; ++a) {
      if (xb) xb[g * 3 + a] = adj[a * np + i];
      if (vb) vb[g * 3 + a] = adj[(3 + a) * np + i];
    }
#pragma unroll
    for (int a = 0; a < 9; ++a) {
      if (Cb) Cb[g * 9 + a] = adj[(6 + a) * np + i];
      if (Fb) Fb[g * 9 + a] = adj[(15 + a) * np + i];
    }
  }
}

// ------------------------------------------------------------------ observations

// One CTA per env: the observation of the live state (row layout in kernels.h).
__global__ void __launch_bounds__(256) k_observe(const EnvDesc* __restrict__ envs, int env0, float* obs, int dim,
                                                 int nsub_max) {
  __shared__ float sh[32];
  const int ei = env0 + blockIdx.x;
  const EnvDesc& e = envs[ei];
  const EnvCtr c = *e.ctr;
  const float* b = e.slots + (long long)c.live * e.block;
  const long long np = e.n_pad;
  const unsigned* meta = reinterpret_cast<const unsigned*>(b + kComp * np);
  const int ns = min(e.n_sub, e.n);
  float* row = obs + (long long)ei * dim;
  float s0 = 0.f, s1 = 0.f, s2 = 0.f;
  for (int i = threadIdx.x; i < e.n; i += blockDim.x) {
    const int id = (int)(meta[i] & kIdMask);
    if (id < ns) {
      const float x0 = b[i], x1 = b[np + i], x2 = b[2 * np + i];
      row[3 * id] = x0;
      row[3 * id + 1] = x1;
      row[3 * id + 2] = x2;
      s0 += x0;
      s1 += x1;
      s2 += x2;
    }
  }
  for (int q = 3 * ns + threadIdx.x; q < 3 * nsub_max; q += blockDim.x) row[q] = 0.f;
  s0 = block_sum(s0, sh);
  s1 = block_sum(s1, sh);
  s2 = block_sum(s2, sh);
  if (threadIdx.x == 0) {
    float* tail = row + 3 * nsub_max;
    const float inv = ns > 0 ? 1.0f / (float)ns : 0.0f;
    tail[0] = s0 * inv;
    tail[1] = s1 * inv;
    tail[2] = s2 * inv;
    const float* q = e.pose + c.live * kPose;
    for (int j = 0; j < 4; ++j)
      tail[3 + j] = e.coll_kind == COLL_CAPSULES ? q[j] : (j < e.n_coll_act ? q[e.act_map[j]] : 0.0f);
    for (int k = 0; k < 3; ++k) tail[7 + k] = e.reward_kind == 2 ? e.rparam[k] : 0.0f;
  }
}

// One CTA per env: adds the adjoint of an observation to the state adjoint (x' and its mean)
// and to the pose adjoint (the action-driven components).
__global__ void __launch_bounds__(256) k_obs_adj(const EnvDesc* __restrict__ envs, int env0, ObsAdj o, int which) {
  if (*o.on == 0) return;
  const int ei = env0 + blockIdx.x;
  const EnvDesc& e = envs[ei];
  const EnvCtr c = *e.ctr;
  const int row_t = which == 0 ? c.rev + 1 : c.rev;
  const float* b = e.slots + (long long)(c.base + row_t) * e.block;
  float* adj = c.par ? e.adj1 : e.adj0;
  const long long np = e.n_pad;
  const unsigned* meta = reinterpret_cast<const unsigned*>(b + kComp * np);
  const int ns = min(e.n_sub, e.n);
  const float* r = o.adj + ((long long)row_t * o.n_tot + ei) * o.dim;
  const float* tail = r + 3 * o.nsub_max;
  const float inv = ns > 0 ? 1.0f / (float)ns : 0.0f;
  const float m0 = tail[0] * inv, m1 = tail[1] * inv, m2 = tail[2] * inv;
  for (int i = threadIdx.x; i < e.n; i += blockDim.x) {
    const int id = (int)(meta[i] & kIdMask);
    if (id < ns) {
      adj[i] += r[3 * id] + m0;
      adj[np + i] += r[3 * id + 1] + m1;
      adj[2 * np + i] += r[3 * id + 2] + m2;
    }
  }
  if (threadIdx.x == 0) {
    if (e.coll_kind == COLL_CAPSULES)
      for (int j = 0; j < 4; ++j) e.acc[ACC_QB + j] += tail[3 + j];
    else
      for (int j = 0; j < e.n_coll_act; ++j) e.acc[ACC_QB + e.act_map[j]] += tail[3 + j];
  }
}

// One thread per environment: the caller's 4-wide pose <-> the slot pose vectors.
// POSE_SET: body 0 of slot 0 from buf, capsule j at buf + j * cap_offset (same angle);
// POSE_KEEP: slot `slot`'s pose vector to slot 0; POSE_GET: body 0 of slot `slot` to buf;
// POSE_GRAD: the gradient with respect to the 4-wide pose (the capsules' pose adjoints summed).
__global__ void k_pose_io(const EnvDesc* __restrict__ envs, int env0, int n_env, int mode, float* buf, int slot) {
  const int ei = env0 + blockIdx.x * blockDim.x + threadIdx.x;
  if (ei >= env0 + n_env) return;
  const EnvDesc& e = envs[ei];
  const int pl = pose_len(e);
  float* b = buf + 4 * (long long)ei;
  if (mode == POSE_SET) {
    for (int j = 0; j < pl / 4; ++j) {
      for (int i = 0; i < 3; ++i) e.pose[4 * j + i] = b[i] + (float)j * e.cap_offset[i];
      e.pose[4 * j + 3] = b[3];
    }
  } else if (mode == POSE_KEEP) {
    for (int i = 0; i < pl; ++i) e.pose[i] = e.pose[slot * kPose + i];
  } else if (mode == POSE_GET) {
    for (int i = 0; i < 4; ++i) b[i] = e.pose[slot * kPose + i];
  } else {
    for (int i = 0; i < 4; ++i) {
      float g = 0.f;
      for (int j = i; j < pl; j += 4) g += e.acc[ACC_QB + j];
      b[i] = g;
    }
  }
}

// ------------------------------------------------------------------ launchers

static std::atomic<long long> g_launches{0};
static TimingHook g_hook;
long long kernel_launch_count() { return g_launches.load(); }
void set_timing_hook(const TimingHook* h) { g_hook = h ? *h : TimingHook{}; }
void count_launches(int n) { g_launches += n; }

struct Timed {  // records the hook's events around one launch of class kc
  int kc;
  cudaStream_t st;
  bool on() const { return g_hook.before && (g_hook.kc == kc || g_hook.kc == -1); }
  Timed(int k, cudaStream_t s) : kc(k), st(s) {
    if (on()) g_hook.before(g_hook.user, kc, st);
  }
  ~Timed() {
    g_launches += 1;
    if (on()) g_hook.after(g_hook.user, kc, st);
  }
};

LaunchScope::LaunchScope(int k, cudaStream_t s) : kc(k), st(s) {
  if (g_hook.before && (g_hook.kc == kc || g_hook.kc == -1)) g_hook.before(g_hook.user, kc, st);
}
LaunchScope::~LaunchScope() {
  g_launches += 1;
  if (g_hook.before && (g_hook.kc == kc || g_hook.kc == -1)) g_hook.after(g_hook.user, kc, st);
}

static inline int nblk(int n, int b) { return (n + b - 1) / b; }

// Seven P2G CTAs per SM need the largest shared-memory carveout (P2G reads nothing twice).
// The gather kernels keep the default, which leaves more L1 for their grid reads: G2P^T, at
// four CTAs per SM, ran 12% slower with the carveout forced to 196 KB (five CTAs) or 228 KB,
// and 6% slower at three CTAs with more L1.
template <int BOX>
static void p2g_carveout(int pct) {
  cudaFuncSetAttribute(k_p2g<MAT_NEOHOOKEAN, BOX>, cudaFuncAttributePreferredSharedMemoryCarveout, pct);
  cudaFuncSetAttribute(k_p2g<MAT_VONMISES, BOX>, cudaFuncAttributePreferredSharedMemoryCarveout, pct);
  cudaFuncSetAttribute(k_p2g<MAT_FLUID, BOX>, cudaFuncAttributePreferredSharedMemoryCarveout, pct);
  cudaFuncSetAttribute(k_p2g<MAT_MUSCLE, BOX>, cudaFuncAttributePreferredSharedMemoryCarveout, pct);
}

static bool scatter_carveout() {
  p2g_carveout<kScBoxSmall>(cudaSharedmemCarveoutMaxShared);
  p2g_carveout<kScBoxLarge>(cudaSharedmemCarveoutMaxShared);
  p2g_carveout<kScBoxWarp>(cudaSharedmemCarveoutMaxShared);
  return true;
}

template <int BOX>
static void p2g_dispatch(const Launch& L, StateRef src, bool use_perm, int k, int rev, const GridTape* skip) {
  const int2* skip_slot = skip ? skip->slot : nullptr;
  const int tT = skip ? skip->T : 0, tS = skip ? skip->S : 0;
  const int pm = use_perm ? 1 : 0;
  switch (L.material) {
    case MAT_NEOHOOKEAN: k_p2g<MAT_NEOHOOKEAN, BOX><<<L.n_items * (kBlock / ScatterThreads<BOX>::value), ScatterThreads<BOX>::value, 0, L.stream>>>(L.envs, L.items, L.item_offset, src, pm, k, rev, L.active, L.active_n, skip_slot, tT, tS); break;
    case MAT_VONMISES: k_p2g<MAT_VONMISES, BOX><<<L.n_items * (kBlock / ScatterThreads<BOX>::value), ScatterThreads<BOX>::value, 0, L.stream>>>(L.envs, L.items, L.item_offset, src, pm, k, rev, L.active, L.active_n, skip_slot, tT, tS); break;
    case MAT_FLUID: k_p2g<MAT_FLUID, BOX><<<L.n_items * (kBlock / ScatterThreads<BOX>::value), ScatterThreads<BOX>::value, 0, L.stream>>>(L.envs, L.items, L.item_offset, src, pm, k, rev, L.active, L.active_n, skip_slot, tT, tS); break;
    default: k_p2g<MAT_MUSCLE, BOX><<<L.n_items * (kBlock / ScatterThreads<BOX>::value), ScatterThreads<BOX>::value, 0, L.stream>>>(L.envs, L.items, L.item_offset, src, pm, k, rev, L.active, L.active_n, skip_slot, tT, tS); break;
  }
}

template <int BOX>
static void g2p_adj_dispatch(const Launch& L, StateRef src, StateRef nxt, bool use_perm, int k) {
  const int pm = use_perm ? 1 : 0;
  switch (L.material) {
    case MAT_NEOHOOKEAN: k_g2p_adj<MAT_NEOHOOKEAN, BOX><<<L.n_items * (kBlock / ScatterThreads<BOX>::value), ScatterThreads<BOX>::value, 0, L.stream>>>(L.envs, L.items, L.item_offset, src, nxt, pm, k); break;
    case MAT_VONMISES: k_g2p_adj<MAT_VONMISES, BOX><<<L.n_items * (kBlock / ScatterThreads<BOX>::value), ScatterThreads<BOX>::value, 0, L.stream>>>(L.envs, L.items, L.item_offset, src, nxt, pm, k); break;
    case MAT_FLUID: k_g2p_adj<MAT_FLUID, BOX><<<L.n_items * (kBlock / ScatterThreads<BOX>::value), ScatterThreads<BOX>::value, 0, L.stream>>>(L.envs, L.items, L.item_offset, src, nxt, pm, k); break;
    default: k_g2p_adj<MAT_MUSCLE, BOX><<<L.n_items * (kBlock / ScatterThreads<BOX>::value), ScatterThreads<BOX>::value, 0, L.stream>>>(L.envs, L.items, L.item_offset, src, nxt, pm, k); break;
  }
}

static void ensure_carveout() {
  static const bool done = scatter_carveout();
  (void)done;
}

void launch_p2g(const Launch& L, StateRef src, bool use_perm, int k, const GridTape* skip_kept) {
  if (L.n_items == 0) return;
  ensure_carveout();
  // a conditional rebuild (all its CTAs exit at once when the tape kept the grid) is timed
  // as "other", so the P2G class holds only full scatters
  Timed tm_(skip_kept ? KC_OTHER : KC_P2G, L.stream);
  const int rev = src.kind == REF_RING || src.kind == REF_REV || src.kind == REF_REVK ? 1 : 0;
  if (L.sc_box == kScBoxLarge) p2g_dispatch<kScBoxLarge>(L, src, use_perm, k, rev, skip_kept);
  else if (L.sc_box == kScBoxWarp) p2g_dispatch<kScBoxWarp>(L, src, use_perm, k, rev, skip_kept);
  else p2g_dispatch<kScBoxSmall>(L, src, use_perm, k, rev, skip_kept);
}

void launch_grid(const Launch& L, int k, GridMode mode, bool rev, const GridTape* record) {
  Timed tm_(KC_GRID, L.stream);
  const GridTape rec = record ? *record : GridTape{nullptr, nullptr, nullptr, nullptr, 0, 0, 0};
  k_grid<<<L.grid_blocks, 256, 0, L.stream>>>(L.envs, L.active, L.active_n, k, (int)mode, rev ? 1 : 0, rec, L.env0);
}

void launch_tape_alloc(const Launch& L, const GridTape& tape, int k) {
  Timed tm_(KC_OTHER, L.stream);
  k_tape_alloc<<<1, 1, 0, L.stream>>>(L.envs, L.env0, tape, k, L.active_n);
}

void launch_restore(const Launch& L, const GridTape& tape, int k) {
  Timed tm_(KC_GRID, L.stream);
  k_restore<<<L.grid_blocks, 256, 0, L.stream>>>(L.envs, L.env0, tape, k, L.active, L.active_n);
}

void launch_g2p(const Launch& L, StateRef src, StateRef dst, bool use_perm, int k) {
  (void)k;
  if (L.n_items == 0) return;
  Timed tm_(KC_G2P, L.stream);
  const int rev = (dst.kind == REF_RING || dst.kind == REF_REVK) ? 1 : 0;
  switch (L.material) {
    case MAT_NEOHOOKEAN: k_g2p<MAT_NEOHOOKEAN><<<L.n_items, kBlock, 0, L.stream>>>(L.envs, L.items, L.item_offset, src, dst, use_perm ? 1 : 0, rev, L.wait_polls, L.g2p_stage); break;
    case MAT_VONMISES: k_g2p<MAT_VONMISES><<<L.n_items, kBlock, 0, L.stream>>>(L.envs, L.items, L.item_offset, src, dst, use_perm ? 1 : 0, rev, L.wait_polls, L.g2p_stage); break;
    case MAT_FLUID: k_g2p<MAT_FLUID><<<L.n_items, kBlock, 0, L.stream>>>(L.envs, L.items, L.item_offset, src, dst, use_perm ? 1 : 0, rev, L.wait_polls, L.g2p_stage); break;
    default: k_g2p<MAT_MUSCLE><<<L.n_items, kBlock, 0, L.stream>>>(L.envs, L.items, L.item_offset, src, dst, use_perm ? 1 : 0, rev, L.wait_polls, L.g2p_stage); break;
  }
}

void launch_step_begin(const Launch& L, const float* act_in, int a_max, bool record) {
  Timed tm_(KC_OTHER, L.stream);
  k_step_begin<<<nblk(L.n_env, 128), 128, 0, L.stream>>>(L.envs, L.env0, L.n_env, act_in, a_max, record ? 1 : 0);
}

void launch_reward_end(const Launch& L, float* reward_out, bool record) {
  Timed tm_(KC_OTHER, L.stream);
  k_reward_end<<<L.n_env, 256, 0, L.stream>>>(L.envs, L.env0, reward_out, record ? 1 : 0);
}

void launch_g2p_adj(const Launch& L, StateRef src, StateRef nxt, bool use_perm, int k) {
  if (L.n_items == 0) return;
  ensure_carveout();
  Timed tm_(KC_G2P_ADJ, L.stream);
  if (L.sc_box == kScBoxLarge) g2p_adj_dispatch<kScBoxLarge>(L, src, nxt, use_perm, k);
  else if (L.sc_box == kScBoxWarp) g2p_adj_dispatch<kScBoxWarp>(L, src, nxt, use_perm, k);
  else g2p_adj_dispatch<kScBoxSmall>(L, src, nxt, use_perm, k);
}

// CTAs of k_grid_adj that fit on the device at once (0 if the runtime cannot say).  The grid
// adjoint's persistent warps stop at this: its registers hold fewer CTAs per SM than the grid
// update's, whose autotuned CTA count the launch shares, and CTAs beyond one resident wave
// only add a tail.
static int grid_adj_resident() {
  int dev = 0, sms = 0, per_sm = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess ||
      cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_grid_adj, 256, 0) != cudaSuccess)
    return 0;
  return sms * per_sm;
}

void launch_grid_adj(const Launch& L, int k) {
  static const int resident = grid_adj_resident();
  Timed tm_(KC_GRID_ADJ, L.stream);
  const int blocks = resident > 0 ? std::min(L.grid_blocks, resident) : L.grid_blocks;
  k_grid_adj<<<blocks, 256, 0, L.stream>>>(L.envs, L.active, L.active_n, k);
}

void launch_p2g_adj(const Launch& L, StateRef src, bool use_perm, int k) {
  (void)k;
  if (L.n_items == 0) return;
  Timed tm_(KC_P2G_ADJ, L.stream);
  switch (L.material) {
    case MAT_NEOHOOKEAN: k_p2g_adj<MAT_NEOHOOKEAN><<<L.n_items, kBlock, 0, L.stream>>>(L.envs, L.items, L.item_offset, src, use_perm ? 1 : 0, k); break;
    case MAT_VONMISES: k_p2g_adj<MAT_VONMISES><<<L.n_items, kBlock, 0, L.stream>>>(L.envs, L.items, L.item_offset, src, use_perm ? 1 : 0, k); break;
    case MAT_FLUID: k_p2g_adj<MAT_FLUID><<<L.n_items, kBlock, 0, L.stream>>>(L.envs, L.items, L.item_offset, src, use_perm ? 1 : 0, k); break;
    default: k_p2g_adj<MAT_MUSCLE><<<L.n_items, kBlock, 0, L.stream>>>(L.envs, L.items, L.item_offset, src, use_perm ? 1 : 0, k); break;
  }
}

void launch_observe(const Launch& L, float* obs, int dim, int nsub_max) {
  Timed tm_(KC_OTHER, L.stream);
  k_observe<<<L.n_env, 256, 0, L.stream>>>(L.envs, L.env0, obs, dim, nsub_max);
}

void launch_obs_adj(const Launch& L, const ObsAdj& o, int which) {
  Timed tm_(KC_OTHER, L.stream);
  k_obs_adj<<<L.n_env, 256, 0, L.stream>>>(L.envs, L.env0, o, which);
}

void launch_bwd_init(const Launch& L, int T) {
  Timed tm_(KC_OTHER, L.stream);
  k_bwd_init<<<nblk(L.n_env, 128), 128, 0, L.stream>>>(L.envs, L.env0, L.n_env, T);
}

void launch_rev_begin(const Launch& L) {
  Timed tm_(KC_OTHER, L.stream);
  k_rev_begin<<<nblk(L.n_env, 128), 128, 0, L.stream>>>(L.envs, L.env0, L.n_env);
}

void launch_reward_adj(const Launch& L, const float* rbar, int n_tot) {
  Timed tm_(KC_OTHER, L.stream);
  k_reward_adj<<<L.n_env, 256, 0, L.stream>>>(L.envs, L.env0, rbar, n_tot);
}

void launch_adj_ref(const Launch& L) { Timed tm_(KC_OTHER, L.stream); k_adj_ref<<<L.n_env, 256, 0, L.stream>>>(L.envs, L.env0); }

void launch_rev_end(const Launch& L, float* act_grad, int n_tot, int a_max) {
  Timed tm_(KC_OTHER, L.stream);
  k_rev_end<<<nblk(L.n_env, 128), 128, 0, L.stream>>>(L.envs, L.env0, L.n_env, act_grad, n_tot, a_max);
}

void launch_set_state(const Launch& L, const float* x, const float* v, const float* C, const float* F,
                      const int* group) {
  if (L.n_items == 0) return;
  Timed tm_(KC_OTHER, L.stream);
  k_set_state<<<L.n_items, 256, 0, L.stream>>>(L.envs, L.items, L.item_offset, x, v, C, F, group);
}

void launch_pose_io(const Launch& L, PoseIo mode, float* buf, int slot) {
  if (L.n_env == 0) return;
  Timed tm_(KC_OTHER, L.stream);
  k_pose_io<<<(L.n_env + 127) / 128, 128, 0, L.stream>>>(L.envs, L.env0, L.n_env, (int)mode, buf, slot);
}

void launch_get_state(const Launch& L, StateRef src, float* x, float* v, float* C, float* F) {
  if (L.n_items == 0) return;
  Timed tm_(KC_OTHER, L.stream);
  k_get_state<<<L.n_items, 256, 0, L.stream>>>(L.envs, L.items, L.item_offset, src, x, v, C, F);
}

void launch_adj_in(const Launch& L, const float* xb, const float* vb, const float* Cb, const float* Fb) {
  if (L.n_items == 0) return;
  Timed tm_(KC_OTHER, L.stream);
  k_adj_in<<<L.n_items, 256, 0, L.stream>>>(L.envs, L.items, L.item_offset, xb, vb, Cb, Fb);
}

void launch_adj_out(const Launch& L, StateRef src, float* xb, float* vb, float* Cb, float* Fb) {
  if (L.n_items == 0) return;
  Timed tm_(KC_OTHER, L.stream);
  k_adj_out<<<L.n_items, 256, 0, L.stream>>>(L.envs, L.items, L.item_offset, src, xb, vb, Cb, Fb);
}

}  // namespace mpm
