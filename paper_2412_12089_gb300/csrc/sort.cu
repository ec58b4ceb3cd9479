// sort.cu -- per-cell binning of particles by a stable LSD radix sort (sm_103a).
//
// MLS-MPM (App. D.3) scatters every particle to the 3x3x3 nodes around its cell base.
// Ordering each environment's particles by (4^3 tile, cell) makes a CTA's particles
// share grid nodes, so P2G can accumulate them in shared memory and G2P hits L1.  The
// key of particle p of environment e is (e << cell_bits) | tile-major cell key; one
// stable radix sort over the whole batch orders every environment at once and never
// moves a particle across environments.  The order is bit-exact: keys come from the
// FP32 positions with each operation rounded separately, ties keep their previous order.
#include <cuda_runtime.h>
#include <stdint.h>

#include "kernels.h"
#include "mpm_math.cuh"
#include "mpm_types.h"

namespace mpm {

constexpr int kSortThreads = 256;
constexpr int kSortItems = 16;                           // keys per thread
constexpr int kSortTile = kSortThreads * kSortItems;     // keys per CTA
constexpr int kRadix = 256;

__device__ __forceinline__ unsigned cell_key(float x, float y, float z, int G, int* oob) {
  const float Gf = (float)G;
  const int bx = cell_base(x, Gf, G, oob), by = cell_base(y, Gf, G, oob), bz = cell_base(z, Gf, G, oob);
  const int TG = G >> 2;
  const unsigned tile = (unsigned)(((bz >> 2) * TG + (by >> 2)) * TG + (bx >> 2));
  return tile * 64u + (unsigned)((bz & 3) * 16 + (by & 3) * 4 + (bx & 3));
}

// Keys and global indices of the live state of every environment in the launch.
__global__ void k_bin_keys(const EnvDesc* __restrict__ envs, const WorkItem* __restrict__ items, int item_off,
                           int cell_bits, unsigned* keys, unsigned* vals, long long poff0) {
  const WorkItem it = items[item_off + blockIdx.x];
  const EnvDesc& e = envs[it.env];
  const EnvCtr* c = e.ctr;
  const float* b = e.slots + (long long)c->live * e.block;
  const long long np = e.n_pad;
  int oob = 0;
  for (int p = threadIdx.x; p < it.count; p += blockDim.x) {
    const int i = it.start + p;
    const unsigned k = cell_key(b[i], b[np + i], b[2 * np + i], e.G, &oob);
    const long long g = e.poff + i - poff0;
    keys[g] = (e.key_env << cell_bits) | k;
    vals[g] = (unsigned)g;
  }
}

// Per-env permutation (local indices) from the sorted global indices.
__global__ void k_bin_perm(const EnvDesc* __restrict__ envs, const WorkItem* __restrict__ items, int item_off,
                           const unsigned* vals, long long poff0) {
  const WorkItem it = items[item_off + blockIdx.x];
  const EnvDesc& e = envs[it.env];
  const EnvCtr* c = e.ctr;
  unsigned* perm = e.perm + (long long)c->live * e.n_pad;
  const long long base = e.poff - poff0;
  for (int p = threadIdx.x; p < it.count; p += blockDim.x) {
    const int i = it.start + p;
    perm[i] = vals[base + i] - (unsigned)base;
  }
}

__global__ void k_plain_keys(const float* x, int n, int G, unsigned* keys, unsigned* vals) {
  int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  int oob = 0;
  keys[i] = cell_key(x[3 * i], x[3 * i + 1], x[3 * i + 2], G, &oob);
  vals[i] = (unsigned)i;
}

// Digit histogram of each CTA's tile: hist[d * nblocks + block].
__global__ void __launch_bounds__(kSortThreads) k_radix_hist(const unsigned* __restrict__ keys, long long n, int shift,
                                                             unsigned* hist) {
  __shared__ unsigned h[kRadix];
  for (int i = threadIdx.x; i < kRadix; i += kSortThreads) h[i] = 0u;
  __syncthreads();
  const long long t0 = (long long)blockIdx.x * kSortTile;
#pragma unroll 4
  for (int it = 0; it < kSortItems; ++it) {
    long long i = t0 + it * kSortThreads + threadIdx.x;
    if (i < n) atomicAdd(&h[(keys[i] >> shift) & (kRadix - 1)], 1u);
  }
  __syncthreads();
  for (int d = threadIdx.x; d < kRadix; d += kSortThreads) hist[(long long)d * gridDim.x + blockIdx.x] = h[d];
}

// Exclusive scan of m counters in one CTA of 1024 threads.
__global__ void __launch_bounds__(1024) k_scan_excl(unsigned* a, long long m) {
  __shared__ unsigned part[1024];
  const long long per = (m + 1023) / 1024;
  const long long b0 = threadIdx.x * per;
  unsigned s = 0;
  for (long long i = 0; i < per; ++i) {
    long long j = b0 + i;
    if (j < m) s += a[j];
  }
  part[threadIdx.x] = s;
  __syncthreads();
  for (int off = 1; off < 1024; off <<= 1) {
    unsigned v = threadIdx.x >= off ? part[threadIdx.x - off] : 0u;
    __syncthreads();
    part[threadIdx.x] += v;
    __syncthreads();
  }
  unsigned run = threadIdx.x ? part[threadIdx.x - 1] : 0u;
  for (long long i = 0; i < per; ++i) {
    long long j = b0 + i;
    if (j < m) {
      unsigned v = a[j];
      a[j] = run;
      run += v;
    }
  }
}

// Multi-CTA exclusive scan: each CTA scans a tile of kScanTile counters in place and
// writes the tile's total; the totals are scanned by k_scan_excl; k_scan_add adds them.
constexpr int kScanTile = 4096;  // counters per scan CTA (1024 threads x 4)

__global__ void __launch_bounds__(1024) k_scan_tiles(unsigned* a, long long m, unsigned* tile_sums) {
  __shared__ unsigned warp_sums[32];
  const long long t0 = (long long)blockIdx.x * kScanTile + threadIdx.x * 4;
  unsigned v[4];
#pragma unroll
  for (int q = 0; q < 4; ++q) v[q] = t0 + q < m ? a[t0 + q] : 0u;
  const unsigned loc = v[0] + v[1] + v[2] + v[3];
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  unsigned incl = loc;
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    const unsigned t = __shfl_up_sync(0xffffffffu, incl, o);
    if (lane >= o) incl += t;
  }
  if (lane == 31) warp_sums[warp] = incl;
  __syncthreads();
  if (warp == 0) {
    unsigned ws = warp_sums[lane], wi = ws;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      const unsigned t = __shfl_up_sync(0xffffffffu, wi, o);
      if (lane >= o) wi += t;
    }
    warp_sums[lane] = wi - ws;  // exclusive
    if (lane == 31) tile_sums[blockIdx.x] = wi;
  }
  __syncthreads();
  unsigned run = warp_sums[warp] + incl - loc;
#pragma unroll
  for (int q = 0; q < 4; ++q) {
    if (t0 + q < m) a[t0 + q] = run;
    run += v[q];
  }
}

__global__ void __launch_bounds__(1024) k_scan_add(unsigned* a, long long m, const unsigned* __restrict__ tile_sums) {
  const unsigned off = tile_sums[blockIdx.x];
  const long long t0 = (long long)blockIdx.x * kScanTile + threadIdx.x * 4;
#pragma unroll
  for (int q = 0; q < 4; ++q)
    if (t0 + q < m) a[t0 + q] += off;
}

long long radix_hist_entries(long long n) {
  const long long m = 256 * ((n + kSortTile - 1) / kSortTile);
  return m + (m + kScanTile - 1) / kScanTile;
}

// Stable scatter.  Warp w of a CTA owns a contiguous run of kSortItems*32 keys of the
// tile and ranks them in order with warp match; warps are then ranked in order, so the
// position of every key is its digit's global offset + its rank in key order.
__global__ void __launch_bounds__(kSortThreads) k_radix_scatter(const unsigned* __restrict__ kin,
                                                                const unsigned* __restrict__ vin, unsigned* kout,
                                                                unsigned* vout, long long n, int shift,
                                                                const unsigned* __restrict__ hist) {
  constexpr int W = kSortThreads / 32;
  __shared__ unsigned cnt[W][kRadix];
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  for (int i = threadIdx.x; i < W * kRadix; i += kSortThreads) (&cnt[0][0])[i] = 0u;
  __syncthreads();
  const long long t0 = (long long)blockIdx.x * kSortTile + (long long)w * (kSortItems * 32);
  const unsigned lt = (1u << lane) - 1u;
  unsigned key[kSortItems], val[kSortItems], rank[kSortItems];
#pragma unroll
  for (int it = 0; it < kSortItems; ++it) {
    const long long i = t0 + it * 32 + lane;
    const bool ok = i < n;
    key[it] = ok ? kin[i] : 0u;
    val[it] = ok ? vin[i] : 0u;
    const unsigned d = ok ? ((key[it] >> shift) & (kRadix - 1)) : (unsigned)kRadix;  // sentinel digit
    const unsigned peers = __match_any_sync(0xffffffffu, d);
    const unsigned r = __popc(peers & lt);
    unsigned before = 0u;
    if (ok) before = cnt[w][d];
    __syncwarp();
    if (ok && r == 0u) cnt[w][d] = before + __popc(peers);
    __syncwarp();
    rank[it] = ok ? before + r : 0xffffffffu;
  }
  __syncthreads();
  for (int d = threadIdx.x; d < kRadix; d += kSortThreads) {
    unsigned run = hist[(long long)d * gridDim.x + blockIdx.x];
    for (int ww = 0; ww < W; ++ww) {
      unsigned c = cnt[ww][d];
      cnt[ww][d] = run;
      run += c;
    }
  }
  __syncthreads();
#pragma unroll
  for (int it = 0; it < kSortItems; ++it) {
    if (rank[it] == 0xffffffffu) continue;
    const unsigned d = (key[it] >> shift) & (kRadix - 1);
    const unsigned pos = cnt[w][d] + rank[it];
    kout[pos] = key[it];
    vout[pos] = val[it];
  }
}

int radix_sort(unsigned** keys, unsigned** vals, long long n, int key_bits, unsigned* hist, cudaStream_t st) {
  int cur = 0;
  if (n <= 1) return cur;
  const int nb = (int)((n + kSortTile - 1) / kSortTile);
  const long long m = (long long)nb * kRadix;
  const int ntiles = (int)((m + kScanTile - 1) / kScanTile);
  unsigned* tile_sums = hist + m;  // radix_hist_entries(n) counters in all
  for (int shift = 0; shift < key_bits; shift += 8) {
    k_radix_hist<<<nb, kSortThreads, 0, st>>>(keys[cur], n, shift, hist);
    if (ntiles == 1) {
      k_scan_excl<<<1, 1024, 0, st>>>(hist, m);
      count_launches(1);
    } else {
      k_scan_tiles<<<ntiles, 1024, 0, st>>>(hist, m, tile_sums);
      k_scan_excl<<<1, 1024, 0, st>>>(tile_sums, ntiles);
      k_scan_add<<<ntiles, 1024, 0, st>>>(hist, m, tile_sums);
      count_launches(3);
    }
    k_radix_scatter<<<nb, kSortThreads, 0, st>>>(keys[cur], vals[cur], keys[cur ^ 1], vals[cur ^ 1], n, shift, hist);
    count_launches(2);
    cur ^= 1;
  }
  return cur;
}

void launch_bin_keys_plain(const float* x, int n, int G, unsigned* keys, unsigned* vals, cudaStream_t st) {
  if (n <= 0) return;
  k_plain_keys<<<(n + 255) / 256, 256, 0, st>>>(x, n, G, keys, vals);
  count_launches(1);
}

// Binning of the live state of the launch's environments into perm[live].
void bin_envs(const Launch& L, long long poff0, long long n_total, int cell_bits, int key_bits, SortScratch& s) {
  if (L.n_items == 0 || n_total == 0) return;
  k_bin_keys<<<L.n_items, 256, 0, L.stream>>>(L.envs, L.items, L.item_offset, cell_bits, s.keys[0], s.vals[0], poff0);
  unsigned* kk[2] = {s.keys[0], s.keys[1]};
  unsigned* vv[2] = {s.vals[0], s.vals[1]};
  int cur = radix_sort(kk, vv, n_total, key_bits, s.hist, L.stream);
  k_bin_perm<<<L.n_items, 256, 0, L.stream>>>(L.envs, L.items, L.item_offset, vv[cur], poff0);
  count_launches(2);
}

}  // namespace mpm
