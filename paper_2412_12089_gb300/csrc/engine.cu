// engine.cu -- step machinery shared by the batch context and the server (see engine.h).
//
// A forward control step (the paper's env.step, Alg. 1): bin the live state, then S substeps
// of P2G -> grid -> G2P, then rewards.  A reverse control step (Sec. 4.1): restore the step's
// checkpoint, recompute its substeps into the ring, then run G2P^T -> grid^T -> P2G^T from the
// last substep to the first.
#include "engine.h"

#include <algorithm>
#include <cmath>
#include <cstdlib>
#include <cstring>
#include <map>
#include <mutex>
#include <tuple>

namespace mpm {

namespace {
size_t align256(size_t b) { return (b + 255) & ~(size_t)255; }

// The autotuner's choices, kept for the process: per (material, grid resolution, bucket of
// particles per cell = round(log2(dx^3 / p_vol))) the scatter shape and G2P's staging, and
// one CTA count for the grid kernels.  Every group built later (batch contexts and the
// server's groups alike) starts from them.
struct TuneKey {
  int material, G, ppc;
  bool operator<(const TuneKey& o) const { return std::tie(material, G, ppc) < std::tie(o.material, o.G, o.ppc); }
};
struct TuneVal {
  int sc_box, g2p_stage;
};
std::mutex g_tune_mu;
std::map<TuneKey, TuneVal> g_tune;
int g_tune_grid_blocks = 0;

TuneKey tune_key(const mpm_env_spec& s) {
  const double dx = 1.0 / (double)s.grid_res;
  const double ppc = dx * dx * dx / std::max((double)s.p_vol, 1e-30);
  return {s.material, s.grid_res, (int)std::floor(std::log2(std::max(ppc, 1.0)) + 0.5)};
}
int bits_for(unsigned long long v) {
  int b = 0;
  while (b < 64 && (v >> b) != 0ull) ++b;
  return b;
}
}  // namespace

namespace {
// Rest data of element e: Dm (edge matrix, row-major) and its determinant, in double.
double rest_edges(const mpm_env_spec& s, long long e, double* Dm) {
  const int* t = s.fem_tets + 4 * e;
  for (int k = 0; k < 3; ++k)
    for (int c = 0; c < 3; ++c) Dm[3 * k + c] = (double)s.fem_rest[3 * t[c + 1] + k] - (double)s.fem_rest[3 * t[0] + k];
  return Dm[0] * (Dm[4] * Dm[8] - Dm[5] * Dm[7]) - Dm[1] * (Dm[3] * Dm[8] - Dm[5] * Dm[6]) +
         Dm[2] * (Dm[3] * Dm[7] - Dm[4] * Dm[6]);
}
}  // namespace

const char* check_spec(const mpm_env_spec& s) {
  if (s.n_particles < 1 || s.n_particles > (int)kIdMask) return "n_particles";
  if (s.grid_res < 8 || s.grid_res > 128 || s.grid_res % 4) return "grid_res";
  if (s.substeps < 1 || s.substeps > 4096) return "substeps";
  if (s.bound < 0 || 2 * s.bound >= s.grid_res) return "bound";
  if (s.material < 0 || s.material > kMatFem) return "material";
  if (s.collider < 0 || s.collider > 4) return "collider";
  if (s.collider == MPM_COLL_CAPSULES) {
    if (s.n_caps < 1 || s.n_caps > kMaxCaps) return "n_caps";
    if (s.n_coll_act != 4 * s.n_caps) return "n_coll_act";
    if (!(s.coll_dims[0] > 0.0f) || !(s.coll_dims[1] >= 0.0f)) return "coll_dims";
  } else {
    if (s.n_coll_act < 0 || s.n_coll_act > 4) return "n_coll_act";
    for (int j = 0; j < s.n_coll_act; ++j)
      if (s.act_map[j] < 0 || s.act_map[j] > 3) return "act_map";
  }
  if (s.n_groups < 0 || s.n_groups > 4094) return "n_groups";
  if (s.n_coll_act + s.n_groups > kMaxAct) return "action dim";
  if (s.reward < 0 || s.reward > 3) return "reward";
  if (s.reward != 0 && s.n_sub < 1) return "n_sub";
  if (!(s.dt > 0.f) || !(s.p_vol > 0.f) || !(s.rho > 0.f)) return "dt/p_vol/rho";
  if (s.reward == 1 && !(s.rparam[0] != 0.f)) return "rparam (h_flat)";
  if ((s.material == 0 || s.material == 1 || s.material == 3 || s.material == kMatFem) &&
      !(s.E > 0.f && s.nu >= 0.f && s.nu < 0.5f))
    return "E/nu";
  if (s.material == kMatFem) {
    if (s.n_particles > kFemMaxVerts) return "n_particles (FEM meshes hold at most 1024 vertices)";
    if (s.collider != MPM_COLL_NONE || s.n_coll_act != 0) return "collider (FEM has none)";
    if (!(s.nu > 0.f)) return "nu (FEM needs lambda > 0)";
    if (s.n_tets < 1 || s.n_tets > kFemMaxElems || !s.fem_tets || !s.fem_rest) return "fem mesh (1..1024 elements)";
    if (!(s.k_damp >= 0.f)) return "k_damp";
    for (long long e = 0; e < s.n_tets; ++e) {
      for (int c = 0; c < 4; ++c)
        if (s.fem_tets[4 * e + c] < 0 || s.fem_tets[4 * e + c] >= s.n_particles) return "fem_tets (vertex index)";
      if (s.fem_group && (s.fem_group[e] < 0 || s.fem_group[e] >= std::max(s.n_groups, 1))) return "fem_group";
      double Dm[9];
      const double det = rest_edges(s, e, Dm);
      if (det == 0.0 || !std::isfinite(det)) return "fem_rest (degenerate element)";
    }
  }
  return nullptr;
}

cudaError_t fem_upload(const mpm_env_spec& s, const EnvDesc& d) {
  if (s.material != kMatFem) return cudaSuccess;
  const long long nt = s.n_tets, nv = s.n_particles;
  std::vector<int4> tet((size_t)nt);
  std::vector<float> dminv((size_t)nt * 9), vol((size_t)nt), inv_mass((size_t)d.n_pad, 0.0f);
  std::vector<int> grp((size_t)nt, 0);
  std::vector<double> mass((size_t)nv, 0.0);
  for (long long e = 0; e < nt; ++e) {
    const int* t = s.fem_tets + 4 * e;
    tet[e] = make_int4(t[0], t[1], t[2], t[3]);
    double Dm[9];
    const double det = rest_edges(s, e, Dm);
    if (det == 0.0 || !std::isfinite(det)) return cudaErrorInvalidValue;
    // inverse by the adjugate: (Dm^-1)_ij = cof(Dm)_ji / det
    const double cof[9] = {Dm[4] * Dm[8] - Dm[5] * Dm[7], Dm[5] * Dm[6] - Dm[3] * Dm[8], Dm[3] * Dm[7] - Dm[4] * Dm[6],
                           Dm[2] * Dm[7] - Dm[1] * Dm[8], Dm[0] * Dm[8] - Dm[2] * Dm[6], Dm[1] * Dm[6] - Dm[0] * Dm[7],
                           Dm[1] * Dm[5] - Dm[2] * Dm[4], Dm[2] * Dm[3] - Dm[0] * Dm[5], Dm[0] * Dm[4] - Dm[1] * Dm[3]};
    for (int i = 0; i < 3; ++i)
      for (int j = 0; j < 3; ++j) dminv[9 * e + 3 * i + j] = (float)(cof[3 * j + i] / det);
    const double V0 = std::fabs(det) / 6.0;
    vol[e] = (float)V0;
    for (int c = 0; c < 4; ++c) mass[t[c]] += 0.25 * (double)s.rho * V0;
    grp[e] = s.fem_group ? s.fem_group[e] : 0;
  }
  for (long long i = 0; i < nv; ++i) inv_mass[i] = mass[i] > 0.0 ? (float)(1.0 / mass[i]) : 0.0f;
  // incidence lists by counting sort (entries in increasing element order)
  const long long ng = std::max(s.n_groups, 1);
  std::vector<int> voff((size_t)d.n_pad + 1, 0), vinc((size_t)(4 * nt)), goff((size_t)ng + 1, 0), ginc((size_t)nt);
  for (long long e = 0; e < nt; ++e) {
    for (int c = 0; c < 4; ++c) voff[s.fem_tets[4 * e + c] + 1] += 1;
    goff[grp[e] + 1] += 1;
  }
  for (long long i = 0; i < (long long)d.n_pad; ++i) voff[i + 1] += voff[i];
  for (long long g = 0; g < ng; ++g) goff[g + 1] += goff[g];
  {
    std::vector<int> vc(voff.begin(), voff.end() - 1), gc(goff.begin(), goff.end() - 1);
    for (long long e = 0; e < nt; ++e) {
      for (int c = 0; c < 4; ++c) vinc[vc[s.fem_tets[4 * e + c]]++] = (int)(4 * e + c);
      ginc[gc[grp[e]]++] = (int)e;
    }
  }
  cudaError_t err;
  if ((err = cudaMemcpy((void*)d.fem_tet, tet.data(), sizeof(int4) * nt, cudaMemcpyHostToDevice))) return err;
  if ((err = cudaMemcpy((void*)d.fem_dminv, dminv.data(), sizeof(float) * 9 * nt, cudaMemcpyHostToDevice))) return err;
  if ((err = cudaMemcpy((void*)d.fem_vol, vol.data(), sizeof(float) * nt, cudaMemcpyHostToDevice))) return err;
  if ((err = cudaMemcpy((void*)d.fem_group, grp.data(), sizeof(int) * nt, cudaMemcpyHostToDevice))) return err;
  if ((err = cudaMemcpy((void*)d.fem_inv_mass, inv_mass.data(), sizeof(float) * d.n_pad, cudaMemcpyHostToDevice)))
    return err;
  if ((err = cudaMemcpy((void*)d.fem_vinc_off, voff.data(), sizeof(int) * voff.size(), cudaMemcpyHostToDevice)))
    return err;
  if ((err = cudaMemcpy((void*)d.fem_vinc, vinc.data(), sizeof(int) * vinc.size(), cudaMemcpyHostToDevice))) return err;
  if ((err = cudaMemcpy((void*)d.fem_ginc_off, goff.data(), sizeof(int) * goff.size(), cudaMemcpyHostToDevice)))
    return err;
  return cudaMemcpy((void*)d.fem_ginc, ginc.data(), sizeof(int) * ginc.size(), cudaMemcpyHostToDevice);
}

EnvLayout env_layout(const mpm_env_spec& s, int n_slots, bool tape, bool own, int T) {
  EnvLayout L;
  L.n_slots = n_slots;
  L.tape = tape;
  L.own = own;
  L.T = own ? T : 0;
  const long long n_pad = ((long long)s.n_particles + 31) / 32 * 32;
  L.n_pad = n_pad;
  const long long block = 25 * n_pad;
  const long long G3 = (long long)s.grid_res * s.grid_res * s.grid_res;
  const long long TG3 = (long long)(s.grid_res / 4) * (s.grid_res / 4) * (s.grid_res / 4);
  const int A = std::max(1, s.n_coll_act + s.n_groups);
  size_t cur = 0;
  L.slots = cur; cur = align256(cur + (size_t)n_slots * block * 4);
  L.ring = cur;  if (tape) cur = align256(cur + (size_t)std::max(s.substeps - 1, 0) * block * 4);
  L.adj = cur;   if (tape) cur = align256(cur + (size_t)2 * kComp * n_pad * 4);
  L.perm = cur;  cur = align256(cur + (size_t)n_slots * n_pad * 4);
  L.grid = cur;  cur = align256(cur + (size_t)(tape ? 4 : 2) * G3 * 16);
  L.tile = cur;  cur = align256(cur + (size_t)TG3 * 4);
  L.pose = cur;  cur = align256(cur + (size_t)n_slots * kPose * 4);
  L.act = cur;   cur = align256(cur + (size_t)n_slots * A * 4);
  if (s.material == kMatFem) {  // element records, Dm^-1, rest volumes, groups, inverse masses, CSRs
    const size_t nt = (size_t)std::max(s.n_tets, 0), ng = (size_t)std::max(s.n_groups, 1);
    L.fem = cur;
    cur = align256(cur + nt * (16 + 36 + 4 + 4) + (size_t)n_pad * 4 + ((size_t)n_pad + 1 + 4 * nt + ng + 1 + nt) * 4);
  }
  if (own) {
    L.acc = cur;       cur = align256(cur + (size_t)(ACC_ACT + A) * 4);
    L.ctr = cur;       cur = align256(cur + sizeof(EnvCtr));
    L.act_env = cur;   cur = align256(cur + (size_t)std::max(T, 1) * A * 4);
    L.rew_env = cur;   cur = align256(cur + (size_t)std::max(T, 1) * 4);
    L.rbar_env = cur;  cur = align256(cur + (size_t)std::max(T, 1) * 4);
    L.agrad_env = cur; cur = align256(cur + (size_t)std::max(T, 1) * A * 4);
    L.xout = cur;      cur = align256(cur + (size_t)s.n_particles * 3 * 4);
  }
  L.total = cur;
  return L;
}

void initial_pose(const mpm_env_spec& s, float* q) {
  for (int i = 0; i < kPose; ++i) q[i] = 0.0f;
  const int bodies = s.collider == MPM_COLL_CAPSULES ? s.n_caps : 1;
  for (int j = 0; j < bodies; ++j) {
    for (int i = 0; i < 3; ++i) q[4 * j + i] = s.pose0[i] + (float)j * (bodies > 1 ? s.cap_offset[i] : 0.0f);
    q[4 * j + 3] = s.pose0[3];
  }
}

void env_fill(EnvDesc& d, const mpm_env_spec& s, const EnvLayout& L, char* base, float* acc, EnvCtr* ctr) {
  memset(&d, 0, sizeof d);
  d.n = s.n_particles;
  d.n_pad = (int)L.n_pad;
  d.G = s.grid_res;
  d.S = s.substeps;
  d.bound = s.bound;
  d.n_slots = L.n_slots;
  d.material = s.material;
  d.coll_kind = s.collider;
  d.n_coll_act = s.n_coll_act;
  d.n_groups = s.n_groups;
  d.reward_kind = s.reward;
  d.n_sub = s.n_sub;
  d.A = s.n_coll_act + s.n_groups;
  for (int j = 0; j < 4; ++j) {
    d.act_map[j] = s.act_map[j];
    d.coll_dims[j] = s.coll_dims[j];
    d.act_scale[j] = s.act_scale[j];
    d.rparam[j] = s.rparam[j];
  }
  d.dt = s.dt;
  d.dx = 1.0f / (float)s.grid_res;
  d.inv_dx = (float)s.grid_res;
  d.p_vol = s.p_vol;
  d.p_mass = s.rho * s.p_vol;
  for (int i = 0; i < 3; ++i) d.gravity[i] = s.gravity[i];
  if (s.material == 0 || s.material == 1 || s.material == 3 || s.material == kMatFem) {
    const double E = s.E, nu = s.nu;
    d.mu = (float)(E / (2.0 * (1.0 + nu)));
    d.lam = (float)(E * nu / ((1.0 + nu) * (1.0 - 2.0 * nu)));
  }
  d.cyl = d.mu > 0.f ? (float)((double)s.c_y * s.yield_stress / (2.0 * d.mu)) : 0.f;
  d.bulk = s.bulk;
  d.visc = s.visc;
  d.act_stress = s.act_stress;
  d.coll_mu = s.coll_mu;
  d.alpha = s.alpha;
  d.ground_mu = s.ground_mu;
  if (s.material == kMatFem) {
    const size_t nt = (size_t)s.n_tets;
    char* f = base + L.fem;
    d.fem_tet = (const int4*)f;
    d.fem_dminv = (const float*)(f + nt * 16);
    d.fem_vol = d.fem_dminv + 9 * nt;
    d.fem_group = (const int*)(d.fem_vol + nt);
    d.fem_inv_mass = (const float*)(d.fem_group + nt);
    d.fem_vinc_off = (const int*)(d.fem_inv_mass + L.n_pad);
    d.fem_vinc = d.fem_vinc_off + L.n_pad + 1;
    d.fem_ginc_off = d.fem_vinc + 4 * nt;
    d.fem_ginc = d.fem_ginc_off + std::max(s.n_groups, 1) + 1;
    d.n_tets = s.n_tets;
    d.k_damp = s.k_damp;
    d.ground_z = s.ground_z;
    d.fem_alpha = (float)(1.0 + 0.75 * (double)d.mu / (double)d.lam);
  }
  if (s.collider == MPM_COLL_CAPSULES) {
    d.n_caps = s.n_caps;
    for (int i = 0; i < 3; ++i) d.cap_offset[i] = s.cap_offset[i];
  }
  d.block = 25 * L.n_pad;
  const long long G3 = (long long)d.G * d.G * d.G;
  d.slots = (float*)(base + L.slots);
  d.ring = L.tape ? (float*)(base + L.ring) : nullptr;
  d.adj0 = L.tape ? (float*)(base + L.adj) : nullptr;
  d.adj1 = L.tape ? d.adj0 + (size_t)kComp * L.n_pad : nullptr;
  d.perm = (unsigned*)(base + L.perm);
  float4* g = (float4*)(base + L.grid);
  d.grid_mp = g;
  d.grid_v = g + G3;
  d.grid_vb = L.tape ? g + 2 * G3 : nullptr;
  d.grid_mpb = L.tape ? g + 3 * G3 : nullptr;
  d.tile = (unsigned*)(base + L.tile);
  d.pose = (float*)(base + L.pose);
  d.act = (float*)(base + L.act);
  if (L.own) {
    d.acc = (float*)(base + L.acc);
    d.ctr = (EnvCtr*)(base + L.ctr);
    d.act_env = (const float*)(base + L.act_env);
    d.rew_env = (float*)(base + L.rew_env);
    d.rbar_env = (const float*)(base + L.rbar_env);
    d.agrad_env = (float*)(base + L.agrad_env);
  } else {
    d.acc = acc;
    d.ctr = ctr;
  }
}

void Group::release() {
  void* ptrs[] = {d_desc, d_items, d_items_env, active, active_n, sort.keys[0], sort.keys[1], sort.vals[0],
                  sort.vals[1], sort.hist, tape.mp, tape.list, tape.slot, tape.cursor, d_fem, keep};
  for (void* p : ptrs)
    if (p) cudaFree(p);
  d_desc = nullptr;
  d_items = d_items_env = nullptr;
  active = nullptr;
  active_n = nullptr;
  sort = SortScratch{};
  desc_cap = items_cap = 0;
  active_cap = hist_cap = 0;
  tape = GridTape{nullptr, nullptr, nullptr, nullptr, 0, 0, 0};
  tape_mp_cap = tape_list_cap = tape_slot_cap = tape_cursor_cap = 0;
  d_fem = nullptr;
  fem_cap = 0;
  keep = nullptr;
  keep_cap = 0;
  keep_n = 0;
}

namespace {
template <typename T>
cudaError_t ensure(T*& p, size_t& cap, size_t n) {
  if (n <= cap && p) return cudaSuccess;
  if (p) cudaFree(p);
  p = nullptr;
  const size_t want = std::max<size_t>(n + n / 4, 16);
  cudaError_t e = cudaMalloc(&p, want * sizeof(T));
  cap = e == cudaSuccess ? want : 0;
  return e;
}
// As ensure, without headroom (for the large grid-tape pool).
template <typename T>
cudaError_t ensure_exact(T*& p, size_t& cap, size_t n) {
  if (n <= cap && p) return cudaSuccess;
  if (p) cudaFree(p);
  p = nullptr;
  cudaError_t e = cudaMalloc(&p, std::max<size_t>(n, 1) * sizeof(T));
  cap = e == cudaSuccess ? std::max<size_t>(n, 1) : 0;
  return e;
}
}  // namespace

cudaError_t group_build(Group& g, const std::vector<EnvDesc>& descs, const std::vector<mpm_env_spec>& specs) {
  g.desc = descs;
  g.spec = specs;
  g.n_envs = (int)descs.size();
  g.S_max = 0;
  g.A_max = 1;
  g.P = 0;
  g.tiles = 0;
  g.fem_envs.clear();
  g.fem_nv_max = g.fem_act_max = g.fem_nt_max = 0;
  int G_max = 8;
  for (int e = 0; e < g.n_envs; ++e) {
    const auto& s = specs[e];
    if (s.material == kMatFem) {
      g.fem_envs.push_back(e);
      g.fem_nv_max = std::max(g.fem_nv_max, s.n_particles);
      g.fem_act_max = std::max(g.fem_act_max, s.n_groups);
      g.fem_nt_max = std::max(g.fem_nt_max, s.n_tets);
    } else {
      g.S_max = std::max(g.S_max, s.substeps);
    }
    g.A_max = std::max(g.A_max, s.n_coll_act + s.n_groups);
    G_max = std::max(G_max, s.grid_res);
    g.desc[e].key_env = (unsigned)e;
    g.desc[e].poff = g.P;
    g.P += s.n_particles;
    g.tiles += (long long)(s.grid_res / 4) * (s.grid_res / 4) * (s.grid_res / 4);
  }
  const unsigned long long max_cell = (unsigned long long)(G_max / 4) * (G_max / 4) * (G_max / 4) * 64ull - 1ull;
  g.cell_bits = bits_for(max_cell);
  g.key_bits = g.cell_bits + bits_for((unsigned long long)std::max(g.n_envs - 1, 0));
  // work items: runs of <= kChunk particles of one environment
  g.items_env.clear();
  g.env_item0.clear();
  g.env_nitems.clear();
  for (int e = 0; e < g.n_envs; ++e) {
    g.env_item0.push_back((int)g.items_env.size());
    int cnt = 0;
    for (int s0 = 0; s0 < specs[e].n_particles; s0 += kChunk) {
      g.items_env.push_back(WorkItem{e, s0, std::min(kChunk, specs[e].n_particles - s0), 0});
      ++cnt;
    }
    g.env_nitems.push_back(cnt);
  }
  // particle kernels are compiled per material: items grouped by material, then by
  // substep count (descending) so substep k launches a prefix of each material's items
  g.items = g.items_env;
  std::stable_sort(g.items.begin(), g.items.end(), [&](const WorkItem& a, const WorkItem& b) {
    const auto &sa = specs[a.env], &sb = specs[b.env];
    if (sa.material != sb.material) return sa.material < sb.material;
    return sa.substeps > sb.substeps;
  });
  // scatter shape (cell capacity of its counting sort) until autotuned; MPM_SCATTER_BOX=
  // 512|1024|256 sets it (tests use it to run every kernel build)
  int box0 = 512;
  if (const char* b = std::getenv("MPM_SCATTER_BOX")) {
    const int v = std::atoi(b);
    for (int b = 0; b < kNScatterBoxes; ++b)
      if (v == kScatterBoxes[b]) box0 = v;
  }
  // test-only: shorten G2P's first bounded wait so that it gives up (the status path)
  g.wait_polls = -1;
  if (const char* wp = std::getenv("MPM_TEST_G2P_WAIT_POLLS")) {
    const int v = std::atoi(wp);
    if (v >= 0) g.wait_polls = v;
  }
  g.mats.clear();
  {
    std::lock_guard<std::mutex> lk(g_tune_mu);
    for (size_t i = 0; i < g.items.size(); ++i) {
      const int mat = specs[g.items[i].env].material;
      if (mat == kMatFem) break;  // FEM items sort last; their envs run the FEM step kernels
      if (g.mats.empty() || g.mats.back().material != mat) {
        g.mats.push_back({mat, (int)i, std::vector<int>(g.S_max + 1, 0), box0});
        // the autotuner's earlier choice for this kind of environment (the variable set by
        // tests to force a shape wins)
        auto t = g_tune.find(tune_key(specs[g.items[i].env]));
        if (t != g_tune.end()) {
          if (!std::getenv("MPM_SCATTER_BOX")) g.mats.back().sc_box = t->second.sc_box;
          g.mats.back().g2p_stage = t->second.g2p_stage;
        }
      }
      auto& m = g.mats.back();
      for (int k = 0; k <= g.S_max; ++k)
        if (specs[g.items[i].env].substeps > k) m.n_gt[k] += 1;
    }
    if (g_tune_grid_blocks > 0) g.grid_blocks = g_tune_grid_blocks;
  }
  cudaError_t e;
  size_t cap;
  cap = g.desc_cap;
  if ((e = ensure(g.d_desc, cap, std::max<size_t>(g.n_envs, 1))) != cudaSuccess) return e;
  g.desc_cap = cap;
  if (g.n_envs && (e = cudaMemcpy(g.d_desc, g.desc.data(), sizeof(EnvDesc) * g.n_envs, cudaMemcpyHostToDevice)))
    return e;
  size_t cap1 = g.items_cap, cap2 = g.items_cap;
  if ((e = ensure(g.d_items, cap1, std::max<size_t>(g.items.size(), 1))) != cudaSuccess) return e;
  if ((e = ensure(g.d_items_env, cap2, std::max<size_t>(g.items.size(), 1))) != cudaSuccess) return e;
  g.items_cap = std::min(cap1, cap2);
  if (!g.items.empty()) {
    if ((e = cudaMemcpy(g.d_items, g.items.data(), sizeof(WorkItem) * g.items.size(), cudaMemcpyHostToDevice))) return e;
    if ((e = cudaMemcpy(g.d_items_env, g.items_env.data(), sizeof(WorkItem) * g.items_env.size(),
                        cudaMemcpyHostToDevice)))
      return e;
  }
  size_t acap = (size_t)g.active_cap;
  if ((e = ensure(g.active, acap, std::max<size_t>((size_t)g.tiles, 1))) != cudaSuccess) return e;
  g.active_cap = (long long)acap;
  if (!g.active_n) {
    if ((e = cudaMalloc(&g.active_n, sizeof(int)))) return e;
    cudaMemset(g.active_n, 0, sizeof(int));
  }
  size_t scap = (size_t)g.sort.cap;
  size_t c0 = scap, c1 = scap, c2 = scap, c3 = scap;
  const size_t P = std::max<size_t>((size_t)g.P, 1);
  if ((e = ensure(g.sort.keys[0], c0, P)) || (e = ensure(g.sort.keys[1], c1, P)) || (e = ensure(g.sort.vals[0], c2, P)) ||
      (e = ensure(g.sort.vals[1], c3, P)))
    return e;
  g.sort.cap = (long long)std::min(std::min(c0, c1), std::min(c2, c3));
  size_t hcap = (size_t)g.hist_cap;
  if ((e = ensure(g.sort.hist, hcap, (size_t)radix_hist_entries((long long)P)))) return e;
  g.hist_cap = (long long)hcap;
  if (!g.fem_envs.empty()) {
    size_t fc = g.fem_cap;
    if ((e = ensure(g.d_fem, fc, g.fem_envs.size())) != cudaSuccess) return e;
    g.fem_cap = fc;
    if ((e = cudaMemcpy(g.d_fem, g.fem_envs.data(), sizeof(int) * g.fem_envs.size(), cudaMemcpyHostToDevice)))
      return e;
  }
  g.tape.cap = 0;
  if (g.want_tape && g.tape_T > 0 && g.tape_budget > 0.0 && g.S_max > 0) {
    // pool: the budget, or 1.5x a generous estimate of the active tiles (P/64 + 1024 per
    // substep: a dense body at eight particles per cell fills about P/130) when that is
    // smaller, so the memory it would not use goes to kept substep states; a substep whose
    // tiles do not fit is rebuilt by P2G.  MPM_GRID_TAPE_TILES caps it (tests make it overflow)
    constexpr double kTileBytes = 64.0 * sizeof(float4) + sizeof(uint2);
    const double est = 1.5 * (double)g.tape_T * g.S_max * ((double)g.P / 64.0 + 1024.0);
    long long tiles = (long long)std::min(g.tape_budget / kTileBytes, est);
    if (const char* cap = std::getenv("MPM_GRID_TAPE_TILES")) {
      const long long c = std::atoll(cap);
      if (c > 0) tiles = std::min(tiles, c);
    }
    tiles = std::max(tiles, 1LL);
    const size_t slots = (size_t)g.tape_T * g.S_max;
    if (ensure_exact(g.tape.mp, g.tape_mp_cap, (size_t)tiles * 64) == cudaSuccess &&
        ensure_exact(g.tape.list, g.tape_list_cap, (size_t)tiles) == cudaSuccess &&
        ensure_exact(g.tape.slot, g.tape_slot_cap, slots) == cudaSuccess &&
        ensure_exact(g.tape.cursor, g.tape_cursor_cap, 1) == cudaSuccess) {
      g.tape.cap = tiles;
      g.tape.T = g.tape_T;
      g.tape.S = g.S_max;
      // no slot is kept until a recorded step writes it
      cudaMemset(g.tape.slot, 0xff, sizeof(int2) * slots);
    } else {
      cudaGetLastError();  // the tape is an optimisation: run without it
    }
  }
  // kept substep states: as many recorded steps as keep_frac of the memory left after the tape
  // (less keep_reserve) holds, at most tape_T; only with a grid tape (which the reverse pass's
  // adjoint substeps still need)
  g.keep_n = 0;
  size_t per_step = 0;  // floats: every particle environment's S - 1 blocks
  for (int i = 0; i < g.n_envs; ++i)
    if (specs[i].material != kMatFem && specs[i].substeps > 1)
      per_step += (size_t)(specs[i].substeps - 1) * (size_t)g.desc[i].block;
  if (g.tape.cap > 0 && g.keep_frac > 0.0 && g.tape_T > 0 && per_step > 0) {
    size_t free_b = 0, total_b = 0;
    if (cudaMemGetInfo(&free_b, &total_b) != cudaSuccess) free_b = 0;
    const double budget = g.keep_frac * std::max(0.0, (double)free_b - g.keep_reserve);
    long long n = std::min<long long>((long long)(budget / (4.0 * (double)per_step)), g.tape_T);
    if (const char* ks = std::getenv("MPM_KEEP_STEPS")) {
      const long long c = std::atoll(ks);
      if (c >= 0) n = std::min(n, c);
    }
    if (n > 0 && ensure_exact(g.keep, g.keep_cap, (size_t)n * per_step) == cudaSuccess)
      g.keep_n = (int)n;
    else
      cudaGetLastError();  // an optimisation too: recompute every step without it
  }
  // environment i's keep_n slots follow those of the environments before it
  size_t off = 0;
  bool any = false;
  for (int i = 0; i < g.n_envs; ++i) {
    EnvDesc& d = g.desc[i];
    const bool k = g.keep_n > 0 && specs[i].material != kMatFem && specs[i].substeps > 1;
    any = any || d.keep_n != 0 || k;
    d.keep = k ? g.keep + off : nullptr;
    d.keep_n = k ? g.keep_n : 0;
    if (k) off += (size_t)g.keep_n * (size_t)(specs[i].substeps - 1) * (size_t)d.block;
  }
  if (any && g.n_envs && (e = cudaMemcpy(g.d_desc, g.desc.data(), sizeof(EnvDesc) * g.n_envs, cudaMemcpyHostToDevice)))
    return e;
  return cudaSuccess;
}

Launch group_launch(const Group& g, cudaStream_t st) {
  Launch L;
  L.envs = g.d_desc;
  L.items = g.d_items;
  L.material = 0;
  L.n_items = (int)g.items.size();
  L.item_offset = 0;
  L.active = g.active;
  L.active_n = g.active_n;
  L.grid_blocks = g.grid_blocks;
  L.env0 = 0;
  L.n_env = g.n_envs;
  L.stream = st;
  L.wait_polls = g.wait_polls;
  return L;
}

Launch env_launch(const Group& g, int e, cudaStream_t st) {
  Launch L = group_launch(g, st);
  L.items = g.d_items_env;
  L.item_offset = g.env_item0[e];
  L.n_items = g.env_nitems[e];
  L.material = g.spec[e].material;
  L.env0 = e;
  L.n_env = 1;
  const int G = g.spec[e].grid_res;
  L.grid_blocks = std::max(1, std::min(152 * 8, (G / 4) * (G / 4) * (G / 4) / 8));
  return L;
}

namespace {

Launch mat_launch(const Launch& L, const MatGroup& m, int k) {
  Launch Lm = L;
  Lm.material = m.material;
  Lm.sc_box = m.sc_box;
  Lm.g2p_stage = m.g2p_stage;
  Lm.item_offset = m.item0;
  Lm.n_items = m.n_gt[std::min(k, (int)m.n_gt.size() - 1)];
  return Lm;
}

// tape: record every substep's grid into the grid tape (recorded steps), or NULL.
// record: the step is recorded; its substep states go to the kept slots when the environment
// keeps states (REF_FWDK), else substeps run in place in the next slot.
void substeps_forward(const Launch& L, const std::vector<MatGroup>& mats, int S, const GridTape* tape,
                      bool record) {
  for (int k = 0; k < S; ++k) {
    cudaMemsetAsync(L.active_n, 0, sizeof(int), L.stream);
    const StateRef src = record ? StateRef{REF_FWDK, k} : StateRef{k == 0 ? REF_LIVE : REF_NEXT, k};
    const StateRef dst = record ? StateRef{REF_FWDK, k + 1} : StateRef{REF_NEXT, k};
    for (auto& m : mats) launch_p2g(mat_launch(L, m, k), src, k == 0, k);
    if (tape) launch_tape_alloc(L, *tape, k);
    launch_grid(L, k, GRID_FWD, false, tape);
    for (auto& m : mats) launch_g2p(mat_launch(L, m, k), src, dst, k == 0, k);
  }
}

// tape: the group's grid tape (the recorded steps kept their grids there), or NULL.
// fem: the FEM environments among L's (device list, count, largest vertex and action counts).
struct FemList {
  const int* list = nullptr;
  int n = 0, nv_max = 0, act_max = 0, nt_max = 0;
};

// kept: the step's substep states were kept by the forward pass, so they are not recomputed.
void reverse_step(const Launch& L, const std::vector<MatGroup>& mats, int S, const float* rbar, float* agrad,
                  int n_tot, int a_max, const GridTape* tape, const ObsAdj* obs, const FemList& fem,
                  bool kept = false) {
  launch_rev_begin(L);
  launch_reward_adj(L, rbar, n_tot);
  if (obs) launch_obs_adj(L, *obs, 0);  // observation of the step's end state
  launch_adj_ref(L);
  launch_fem_reverse(L, fem.list, fem.n, fem.nv_max, fem.act_max, fem.nt_max);
  // recompute substep states 1..S-1 into the ring (envs with S > k + 1), unless the forward
  // pass kept them; the grid of each substep comes from the tape when it was kept, else P2G
  // rebuilds it
  for (int k = 0; !kept && k + 1 < S; ++k) {
    cudaMemsetAsync(L.active_n, 0, sizeof(int), L.stream);
    const StateRef src{REF_REVK, k};
    const StateRef dst{REF_REVK, k + 1};
    if (tape) launch_restore(L, *tape, k);
    for (auto& m : mats) launch_p2g(mat_launch(L, m, k + 1), src, k == 0, k, tape);
    launch_grid(L, k, GRID_FWD, true);
    for (auto& m : mats) launch_g2p(mat_launch(L, m, k + 1), src, dst, k == 0, k);
  }
  // adjoint substeps, last to first (envs with S > k)
  for (int k = S - 1; k >= 0; --k) {
    cudaMemsetAsync(L.active_n, 0, sizeof(int), L.stream);
    const StateRef src{REF_REVK, k};
    if (tape) launch_restore(L, *tape, k);
    for (auto& m : mats) launch_p2g(mat_launch(L, m, k), src, k == 0, k, tape);
    launch_grid(L, k, GRID_KEEP, true);
    // the end state of substep k (REF_REVK k+1): its kept or ring block for envs with
    // S > k+1, the step's end checkpoint for envs whose last substep is k
    for (auto& m : mats) launch_g2p_adj(mat_launch(L, m, k), src, StateRef{REF_REVK, k + 1}, k == 0, k);
    launch_grid_adj(L, k);
    for (auto& m : mats) launch_p2g_adj(mat_launch(L, m, k), src, k == 0, k);
  }
  launch_rev_end(L, agrad, n_tot, a_max);
}

}  // namespace

cudaError_t autotune_scatter(Group& g, cudaStream_t st, int trials, TuneTimes* times) {
  if (g.n_envs == 0) return cudaSuccess;
  trials = std::max(trials, 1);
  Launch L = group_launch(g, st);
  bin_envs(L, 0, g.P, g.cell_bits, g.key_bits, g.sort);  // permutation of the live state
  cudaEvent_t e0 = nullptr, e1 = nullptr;
  cudaError_t err = cudaEventCreate(&e0);
  if (err == cudaSuccess) err = cudaEventCreate(&e1);
  if (times) {
    times->p2g.assign(g.mats.size(), std::vector<float>());
    times->g2p.assign(g.mats.size(), std::vector<float>());
    times->grid.clear();
  }
  auto elapsed = [&](float* t_ms) {
    cudaError_t e = cudaEventSynchronize(e1);
    if (e == cudaSuccess) e = cudaEventElapsedTime(t_ms, e0, e1);
    return e;
  };
  // scatter shape, per material: P2G of the live state, then the grid update clears the grid
  for (size_t mi = 0; mi < g.mats.size() && err == cudaSuccess; ++mi) {
    MatGroup& m = g.mats[mi];
    float best = 0.0f;
    int best_box = m.sc_box;
    for (int bi = 0; bi < kNScatterBoxes && err == cudaSuccess; ++bi) {
      const int box = kScatterBoxes[bi];
      float best_t = 3.4e38f;
      for (int t = 0; t <= trials && err == cudaSuccess; ++t) {
        cudaMemsetAsync(L.active_n, 0, sizeof(int), st);
        Launch Lm = mat_launch(L, m, 0);
        Lm.sc_box = box;
        cudaEventRecord(e0, st);
        launch_p2g(Lm, StateRef{REF_LIVE, 0}, true, 0);
        cudaEventRecord(e1, st);
        launch_grid(L, 0, GRID_FWD, false);  // consumes and clears the grid and tile flags
        float t_ms = 0.0f;
        err = elapsed(&t_ms);
        if (t > 0) best_t = std::min(best_t, t_ms);
      }
      const float mean = best_t;  // the fastest trial: host-side delays before a launch only add
      if (times) times->p2g[mi].push_back(mean);
      if (bi == 0 || mean < best) {
        best = mean;
        best_box = box;
      }
    }
    if (err == cudaSuccess) m.sc_box = best_box;
  }
  // grid-update CTAs: P2G of every material, then the timed grid update with each choice
  {
    float best = 0.0f;
    int best_blocks = g.grid_blocks;
    for (int ci = 0; ci < 4 && err == cudaSuccess; ++ci) {
      float best_t = 3.4e38f;
      for (int t = 0; t <= trials && err == cudaSuccess; ++t) {
        cudaMemsetAsync(L.active_n, 0, sizeof(int), st);
        for (auto& m : g.mats) launch_p2g(mat_launch(L, m, 0), StateRef{REF_LIVE, 0}, true, 0);
        Launch Lg = L;
        Lg.grid_blocks = kGridBlockChoices[ci];
        cudaEventRecord(e0, st);
        launch_grid(Lg, 0, GRID_FWD, false);
        cudaEventRecord(e1, st);
        float t_ms = 0.0f;
        err = elapsed(&t_ms);
        if (t > 0) best_t = std::min(best_t, t_ms);
      }
      const float mean = best_t;  // the fastest trial: host-side delays before a launch only add
      if (times) times->grid.push_back(mean);
      if (ci == 0 || mean < best) {
        best = mean;
        best_blocks = kGridBlockChoices[ci];
      }
    }
    if (err == cudaSuccess) g.grid_blocks = best_blocks;
    L.grid_blocks = g.grid_blocks;
  }
  // G2P staging, per material: one P2G + grid update gives grid velocities of the live
  // state, then G2P reads the live state in place (binned order after any control step) and
  // writes the first block of the substep ring (scratch between reverse passes), with and
  // without the bulk-copy staging.  Only for contexts whose environments all keep a ring
  // (a checkpoint tape) and run more than one substep; otherwise the default (staging) stays.
  bool ring = true;
  for (const auto& d : g.desc) ring = ring && d.ring != nullptr && d.S > 1;
  if (err == cudaSuccess && ring) {
    cudaMemsetAsync(L.active_n, 0, sizeof(int), st);
    for (auto& m : g.mats) launch_p2g(mat_launch(L, m, 0), StateRef{REF_LIVE, 0}, true, 0);
    launch_grid(L, 0, GRID_FWD, false);  // grid velocities of the active tiles; (m, p) cleared
    for (size_t mi = 0; mi < g.mats.size() && err == cudaSuccess; ++mi) {
      MatGroup& m = g.mats[mi];
      float best = 0.0f;
      int best_stage = m.g2p_stage;
      for (int sg = 0; sg < 2 && err == cudaSuccess; ++sg) {
        float best_t = 3.4e38f;
        for (int t = 0; t <= trials && err == cudaSuccess; ++t) {
          Launch Lm = mat_launch(L, m, 1);
          Lm.g2p_stage = sg;
          cudaEventRecord(e0, st);
          launch_g2p(Lm, StateRef{REF_LIVE, 0}, StateRef{REF_RING, 1}, false, 1);
          cudaEventRecord(e1, st);
          float t_ms = 0.0f;
          err = elapsed(&t_ms);
          if (t > 0) best_t = std::min(best_t, t_ms);
        }
        const float mean = best_t;  // the fastest trial: host-side delays before a launch only add
        if (times) times->g2p[mi].push_back(mean);
        if (sg == 0 || mean < best) {
          best = mean;
          best_stage = sg;
        }
      }
      if (err == cudaSuccess) m.g2p_stage = best_stage;
    }
  }
  if (err == cudaSuccess) {  // keep the choices for groups built later in the process
    std::lock_guard<std::mutex> lk(g_tune_mu);
    for (const auto& m : g.mats) g_tune[tune_key(g.spec[g.items[m.item0].env])] = {m.sc_box, m.g2p_stage};
    g_tune_grid_blocks = g.grid_blocks;
  }
  if (e0) cudaEventDestroy(e0);
  if (e1) cudaEventDestroy(e1);
  return err;
}

void enqueue_forward(Group& g, cudaStream_t st, bool record, const float* act_in, int a_max, float* rew,
                     bool per_env) {
  if (g.n_envs == 0) return;
  if (!per_env) {
    Launch L = group_launch(g, st);
    launch_step_begin(L, act_in, a_max, record);
    launch_fem_forward(L, g.d_fem, (int)g.fem_envs.size(), g.fem_nv_max, g.fem_nt_max);
    if (g.S_max > 0) {
      bin_envs(L, 0, g.P, g.cell_bits, g.key_bits, g.sort);
      substeps_forward(L, g.mats, g.S_max, record && g.tape.cap > 0 ? &g.tape : nullptr, record);
    }
    launch_reward_end(L, rew, record);
    return;
  }
  // baseline path: every stage launched once per environment
  int fem_i = 0;
  for (int e = 0; e < g.n_envs; ++e) {
    Launch L = env_launch(g, e, st);
    if (g.spec[e].material == kMatFem) {
      launch_step_begin(L, act_in, a_max, record);
      launch_fem_forward(L, g.d_fem + fem_i++, 1, g.spec[e].n_particles, g.spec[e].n_tets);
      launch_reward_end(L, rew, record);
      continue;
    }
    const int S = g.spec[e].substeps;
    std::vector<MatGroup> one{{g.spec[e].material, g.env_item0[e], std::vector<int>(S + 1, g.env_nitems[e])}};
    one[0].n_gt[S] = 0;
    launch_step_begin(L, act_in, a_max, record);
    bin_envs(L, g.desc[e].poff, g.spec[e].n_particles, g.cell_bits, g.cell_bits, g.sort);
    substeps_forward(L, one, S, nullptr, record);
    launch_reward_end(L, rew, record);
  }
}

void enqueue_reverse(Group& g, cudaStream_t st, const float* rbar, float* agrad, int n_tot, int a_max, bool per_env,
                     const ObsAdj* obs, bool kept) {
  if (g.n_envs == 0) return;
  if (!per_env) {
    FemList fem{g.d_fem, (int)g.fem_envs.size(), g.fem_nv_max, g.fem_act_max, g.fem_nt_max};
    reverse_step(group_launch(g, st), g.mats, g.S_max, rbar, agrad, n_tot, a_max, g.tape.cap > 0 ? &g.tape : nullptr,
                 obs, fem, kept && g.keep_n > 0);
    return;
  }
  int fem_i = 0;
  for (int e = 0; e < g.n_envs; ++e) {
    if (g.spec[e].material == kMatFem) {
      FemList fem{g.d_fem + fem_i++, 1, g.spec[e].n_particles, g.spec[e].n_groups, g.spec[e].n_tets};
      reverse_step(env_launch(g, e, st), {}, 0, rbar, agrad, n_tot, a_max, nullptr, obs, fem);
      continue;
    }
    const int S = g.spec[e].substeps;
    std::vector<MatGroup> one{{g.spec[e].material, g.env_item0[e], std::vector<int>(S + 1, g.env_nitems[e])}};
    one[0].n_gt[S] = 0;
    reverse_step(env_launch(g, e, st), one, S, rbar, agrad, n_tot, a_max, nullptr, obs, FemList{});
  }
}

}  // namespace mpm
