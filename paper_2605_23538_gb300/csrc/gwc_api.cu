// gwc_api.cu -- the C ABI (include/gwc.h): validation, device layout, launch sequences.
//
// Device layout built by gwc_create:
//   samples      float4 {m1_det, m2_det, d_L, ln pi_PE} + int32 pixel, sorted by event
//                and, within an event, by (pixel, d_L) (a chunk touches few LOS rows, and
//                a warp's lanes read neighbouring table nodes and LOS cells)
//   injections   float4 {m1_det, m2_det, d_L, ln p_draw}, sorted by d_L, then each block
//                of 256 by m1_det (lanes outside the mass support gather into whole warps)
//   LOS table    [n_pix][n_z] float (or bfloat16); the pixel mean in float and double
//   work items   runs of <= chunk samples of one event (events split evenly), then runs
//                of injections; launched largest first
// Per call (sized for max_K at create, so calls allocate nothing):
//   per-Lambda constants and tables, the batch's order by H0, and the partial sums
//   [K][items][PSTRIDE floats].
#include <algorithm>
#include <cmath>
#include <cstdio>
#include <cstring>
#include <map>
#include <mutex>
#include <new>
#include <set>
#include <string>
#include <vector>

#include "../../include/gwc.h"
#include "gwc_kernels.h"

using namespace gwc;

namespace {

constexpr uint32_t MAGIC = 0x67776331u;   // "gwc1"
constexpr size_t INJ_BLOCK = 256;          // injections sorted by m1_det within blocks of this size
thread_local std::string t_err;
std::mutex g_mu;
std::set<const gwc_ctx*> g_live;

}  // namespace

void gwc::set_thread_error(const std::string& msg) { t_err = msg; }

struct gwc_ctx {
  uint32_t magic = MAGIC;
  int device = 0;
  gwc_options opt{};
  int32_t n_events = 0;
  int64_t n_samples = 0, n_inj = 0;
  double n_draw = 0.0;
  int32_t n_pix = 0, n_z = 0;
  double z_max = 0.0;
  bool bf16 = false;
  bool mp = false;      // multi-peak mass model
  int np = NP;          // Lambda entries per point of the mass model (13 or 16)
  int32_t n_items = 0, inj_item0 = 0;
  int tstride = 0;
  int64_t device_bytes = 0;
  // device memory
  float4* smp = nullptr;
  int32_t* pix = nullptr;
  float4* inj = nullptr;
  void* los = nullptr;
  float* pbar32 = nullptr;
  double* pbar64 = nullptr;
  Item* items = nullptr;
  int32_t* sched = nullptr;
  int32_t* ev_item0 = nullptr;
  double* ln_ev_n = nullptr;      // ln N_i per event (the merge's normaliser)
  LamF* lf = nullptr;
  LamD* ld = nullptr;
  float* tables = nullptr;
  float* partials = nullptr;
  int32_t* counter = nullptr;   // work counter of the persistent fused kernel
  int32_t* order = nullptr;     // [max_K] the batch's points ordered by H0 (the prologue writes it)
  int64_t items_cap = 0;        // work items the items/sched/partials buffers hold
  int live_recordings = 0;      // graphs and HMC objects recorded on this context
  // KDE form of the event term: (event, pixel) groups, built at create; device copies,
  // the LOS prior on the KDE grid and the partial buffer made on first use
  std::vector<KdeGroup> h_groups;
  std::vector<int32_t> h_ev_group0;
  KdeGroup* kde_groups = nullptr;
  int32_t* kde_ev_group0 = nullptr;
  int32_t* kde_sched_inj = nullptr;
  float* kde_pgrid = nullptr;
  int kde_G = 0;
  float* kde_partials = nullptr;
  int64_t kde_stride = 0;
  float2* kde_lm = nullptr;     // log2 masses of every sample
  uint64_t serial = 0;          // distinguishes contexts that reuse an address
  std::vector<int64_t> h_offsets;   // event offsets (for re-splitting the work items)
  int n_sms = 0;
  std::map<uint64_t, int> occupancy;   // fused-kernel CTAs per SM by geometry
  bool prof_off = false;               // recording a graph or autotuning: no profiling events
  // host-call staging
  double* d_lam = nullptr;
  double* d_out = nullptr;      // lnL_event, neff_event, ln_xi, neff_sel, lnL_total, grad
  int32_t* d_flags = nullptr;
  double* h_lam = nullptr;      // pinned
  double* h_out = nullptr;      // pinned: lnL_total[K], grad[K][np]
  int32_t* h_flags = nullptr;   // pinned
  // plain path scratch (allocated on first use)
  int32_t* sample_item = nullptr;
  float* plain_lw = nullptr;
  float* plain_tg = nullptr;
  std::vector<int32_t> h_sample_item;
  // profiling: a ring of event quadruples (start, after prologue, after samples, after merge)
  std::vector<cudaEvent_t> prof_ev;
  int prof_used = 0;
  double prof_ms[3] = {0.0, 0.0, 0.0};
  int64_t prof_calls = 0;
  std::string err;
};

namespace {

gwc_status fail(gwc_ctx* c, gwc_status s, const std::string& msg) {
  if (c) c->err = msg; else t_err = msg;
  t_err = msg;
  return s;
}

gwc_status cuda_fail(gwc_ctx* c, cudaError_t e, const char* what) {
  return fail(c, GWC_E_CUDA, std::string(what) + ": " + cudaGetErrorString(e));
}

bool live(const gwc_ctx* c) {
  std::lock_guard<std::mutex> g(g_mu);
  return c && g_live.count(c) && c->magic == MAGIC;
}

template <class T>
cudaError_t dalloc(gwc_ctx* c, T** p, size_t n) {
  *p = nullptr;
  if (n == 0) n = 1;
  cudaError_t e = cudaMalloc(reinterpret_cast<void**>(p), n * sizeof(T));
  if (e == cudaSuccess) c->device_bytes += (int64_t)(n * sizeof(T));
  return e;
}

void free_all(gwc_ctx* c) {
  for (cudaEvent_t e : c->prof_ev) cudaEventDestroy(e);
  c->prof_ev.clear();
  void* dev[] = {c->smp, c->pix, c->inj, c->los, c->pbar32, c->pbar64, c->items, c->sched,
                 c->ev_item0, c->ln_ev_n, c->lf, c->ld, c->tables, c->partials, c->counter, c->order, c->d_lam, c->d_out,
                 c->kde_groups, c->kde_ev_group0, c->kde_sched_inj, c->kde_pgrid, c->kde_partials, c->kde_lm,
                 c->d_flags, c->sample_item, c->plain_lw, c->plain_tg};
  for (void* p : dev)
    if (p) cudaFree(p);
  if (c->h_lam) cudaFreeHost(c->h_lam);
  if (c->h_out) cudaFreeHost(c->h_out);
  if (c->h_flags) cudaFreeHost(c->h_flags);
}

constexpr int PROF_SLOTS = 256;
// one warp per Lambda point: warps then claim points from a shared counter, so uneven
// per-point work (cuts, early rejections) leaves no warp idle at the unit's barrier
constexpr int DEFAULT_LAMBDA_GROUP = 1;
// warps sharing one Lambda point for a batch of K: the context's setting, else the
// default, except that a batch of fewer than 8 points takes the largest power of two
// <= 8 / K, so that a small batch (K = 1 in an HMC chain) still keeps every warp of a
// CTA working (with one warp per point, a K = 1 unit would run on one warp of eight)
int group_for(const gwc_ctx* c, int K) {
  if (c->opt.lambda_group > 0) return c->opt.lambda_group;
  int g = DEFAULT_LAMBDA_GROUP;
  while (g < WARPS && 2 * g * K <= WARPS) g *= 2;
  return g;
}
// the whole batch in one tile (up to 256 points): each staged chunk serves every point,
// and a warp's share of points is large enough that the warps finish a unit together
constexpr int DEFAULT_LAMBDA_TILE = MAX_SLAB;

// fold the recorded quadruples into the sums (waits for them)
cudaError_t prof_drain(gwc_ctx* c) {
  for (int q = 0; q < c->prof_used; ++q) {
    cudaEvent_t* e = &c->prof_ev[(size_t)q * 4];
    cudaError_t r = cudaEventSynchronize(e[3]);
    if (r != cudaSuccess) return r;
    for (int st = 0; st < 3; ++st) {
      float ms = 0.f;
      r = cudaEventElapsedTime(&ms, e[st], e[st + 1]);
      if (r != cudaSuccess) return r;
      c->prof_ms[st] += ms;
    }
    ++c->prof_calls;
  }
  c->prof_used = 0;
  return cudaSuccess;
}

// event of stage boundary b (0..3) of the current call, or nullptr when not profiling
cudaEvent_t prof_event(gwc_ctx* c, int b) {
  if (c->prof_ev.empty()) return nullptr;
  return c->prof_ev[(size_t)c->prof_used * 4 + b];
}

cudaError_t prof_mark(gwc_ctx* c, int b, cudaStream_t s) {
  if (c->prof_ev.empty() || c->prof_off) return cudaSuccess;
  if (b == 0 && c->prof_used == PROF_SLOTS) {
    cudaError_t r = prof_drain(c);
    if (r != cudaSuccess) return r;
  }
  cudaError_t r = cudaEventRecord(prof_event(c, b), s);
  if (b == 3 && r == cudaSuccess) ++c->prof_used;
  return r;
}

uint16_t to_bf16(float f) {   // round to nearest even
  uint32_t u;
  std::memcpy(&u, &f, 4);
  const uint32_t lsb = (u >> 16) & 1u;
  u += 0x7fffu + lsb;
  return (uint16_t)(u >> 16);
}
float from_bf16(uint16_t h) {
  const uint32_t u = (uint32_t)h << 16;
  float f;
  std::memcpy(&f, &u, 4);
  return f;
}

bool finite_all(const float* a, int64_t n) {
  for (int64_t i = 0; i < n; ++i)
    if (!std::isfinite(a[i])) return false;
  return true;
}

void split_items(int64_t begin, int64_t count, int chunk, int32_t kind, std::vector<Item>& out) {
  const int64_t parts = (count + chunk - 1) / chunk;
  for (int64_t p = 0; p < parts; ++p) {
    const int64_t a = begin + count * p / parts, b = begin + count * (p + 1) / parts;
    out.push_back(Item{a, (int32_t)(b - a), kind});
  }
}

// the work items of a chunk size: each event's samples split evenly into runs of at
// most chunk, then the injections; the schedule lists them largest first
struct ItemLayout {
  std::vector<Item> items;
  std::vector<int32_t> sched, ev_item0, sample_item;
  int32_t inj_item0 = 0;
};

bool make_items(const int64_t* offsets, int32_t ne, int64_t ns, int64_t ni, int chunk, ItemLayout& L) {
  L = ItemLayout();
  L.ev_item0.assign((size_t)ne + 1, 0);
  for (int32_t e = 0; e < ne; ++e) {
    L.ev_item0[(size_t)e] = (int32_t)L.items.size();
    split_items(offsets[e], offsets[e + 1] - offsets[e], chunk, 0, L.items);
  }
  L.ev_item0[(size_t)ne] = (int32_t)L.items.size();
  L.inj_item0 = (int32_t)L.items.size();
  split_items(0, ni, chunk, 1, L.items);
  if (L.items.size() > 0x7fffffffu) return false;
  const int32_t n = (int32_t)L.items.size();
  L.sched.resize((size_t)n);
  for (int32_t i = 0; i < n; ++i) L.sched[(size_t)i] = i;
  std::stable_sort(L.sched.begin(), L.sched.end(),
                   [&](int32_t a, int32_t b) { return L.items[(size_t)a].count > L.items[(size_t)b].count; });
  L.sample_item.assign((size_t)(ns + ni), 0);
  for (int32_t i = 0; i < n; ++i) {
    const Item& it = L.items[(size_t)i];
    const int64_t base = it.kind == 1 ? ns + it.begin : it.begin;
    for (int32_t q = 0; q < it.count; ++q) L.sample_item[(size_t)(base + q)] = i;
  }
  return true;
}

// launch geometry of the fused kernel for a batch of K points
void fused_geometry(const gwc_ctx* c, int K, int& slab, int& n_slabs) {
  slab = c->opt.lambda_tile > 0 ? c->opt.lambda_tile : DEFAULT_LAMBDA_TILE;
  const int group = group_for(c, K);
  slab = std::max(1, std::min(std::min(slab, K), std::min(MAX_SLAB, MAX_SLAB_GROUP / group)));
  n_slabs = (K + slab - 1) / slab;
}

gwc_status check_call(gwc_ctx* c, int32_t K, const void* lam, const void* lnL_event,
                      const void* neff_event, const void* ln_xi, const void* neff_sel,
                      const void* lnL_total, const void* flags) {
  if (!live(c)) return fail(nullptr, GWC_E_INVALID, "invalid or destroyed context");
  if (K < 1 || K > c->opt.max_K)
    return fail(c, GWC_E_INVALID, "K must be in [1, max_K] (max_K = " + std::to_string(c->opt.max_K) + ")");
  if (!lam || !ln_xi || !neff_sel || !lnL_total || !flags)
    return fail(c, GWC_E_INVALID, "NULL Lambda or output pointer");
  if (c->n_events > 0 && (!lnL_event || !neff_event))
    return fail(c, GWC_E_INVALID, "NULL per-event output pointer");
  if (cudaSetDevice(c->device) != cudaSuccess) return fail(c, GWC_E_CUDA, "cudaSetDevice failed");
  return GWC_OK;
}

gwc_status run_prologue(gwc_ctx* c, int K, const double* d_lambda, bool grad, cudaStream_t s,
                        int32_t* counter = nullptr) {
  ProArgs pa;
  pa.counter = counter;
  pa.order = c->order;
  pa.lam = d_lambda;
  pa.nx = c->opt.n_x_table;
  pa.nz = c->n_z;
  pa.zmax = c->z_max;
  pa.pbar64 = c->pbar64;
  pa.lf = c->lf;
  pa.ld = c->ld;
  pa.tables = c->tables;
  pa.tstride = c->tstride;
  pa.want_grad = grad ? 1 : 0;
  pa.mp = c->mp ? 1 : 0;
  cudaError_t e = launch_prologue(pa, K, s);
  if (e != cudaSuccess) return cuda_fail(c, e, "prologue launch");
  return GWC_OK;
}

gwc_status run_merge(gwc_ctx* c, int K, int P, bool grad, double* lnL_event, double* neff_event,
                     double* ln_xi, double* neff_sel, double* lnL_total, int32_t* flags,
                     double* grad_total, cudaStream_t s, double* sum_events = nullptr,
                     double* grad_events = nullptr, double* grad_ln_xi = nullptr) {
  MergeArgs ma;
  ma.mp = c->mp ? 1 : 0;
  ma.sum_events = sum_events;
  ma.grad_events = grad_events;
  ma.grad_ln_xi = grad_ln_xi;
  ma.partials = c->partials;
  ma.n_items = c->n_items;
  ma.P = P;
  ma.ev_item0 = c->ev_item0;
  ma.n_events = c->n_events;
  ma.inj_item0 = c->inj_item0;
  ma.ln_ev_n = c->ln_ev_n;
  ma.ln_n_draw = std::log(c->n_draw);
  ma.ld = c->ld;
  ma.neff_min_event = c->opt.neff_min_event;
  ma.neff_min_sel = c->opt.neff_min_sel;
  ma.lnL_event = lnL_event;
  ma.neff_event = neff_event;
  ma.ln_xi = ln_xi;
  ma.neff_sel = neff_sel;
  ma.lnL_total = lnL_total;
  ma.flags = flags;
  ma.grad_total = grad_total;
  cudaError_t e = launch_merge(ma, K, grad, s);
  if (e != cudaSuccess) return cuda_fail(c, e, "merge launch");
  return GWC_OK;
}

// the persistent fused kernel over the n_sched items listed in sched, writing partial
// slot slot0 + item of a [K][stride][PSTRIDE] buffer
gwc_status launch_fused_items(gwc_ctx* c, int32_t K, bool grad, const int32_t* sched, int n_sched,
                              float* partials, int64_t stride, int64_t slot0, cudaStream_t s) {
  int slab, n_slabs;
  fused_geometry(c, K, slab, n_slabs);
  FusedArgs fa;
  fa.smp = c->smp;
  fa.pix = c->pix;
  fa.inj = c->inj;
  fa.los = c->los;
  fa.pbar32 = c->pbar32;
  fa.nz = c->n_z;
  fa.nx = c->opt.n_x_table;
  fa.items = c->items;
  fa.sched = sched;
  fa.n_items = c->n_items;
  fa.n_slabs = n_slabs;
  fa.slab = slab;
  fa.group = group_for(c, K);
  fa.K = K;
  fa.chunk = c->opt.chunk;
  fa.lf = c->lf;
  fa.tables = c->tables;
  fa.tstride = c->tstride;
  fa.partials = partials;
  fa.counter = c->counter;
  fa.order = c->order;
  fa.n_sched = n_sched;
  fa.stride = (int)stride;
  fa.slot0 = (int)slot0;
  fa.mp = c->mp ? 1 : 0;
  const long long units = (long long)n_sched * n_slabs;
  if (units > 0x7fffffffLL) return fail(c, GWC_E_INVALID, "work grid too large");
  // persistent launch: as many CTAs as fit on the GPU at once, each taking units in
  // schedule order (largest items first) from the counter
  const bool kahan = c->opt.accum == 1;
  const uint64_t key = ((uint64_t)fa.chunk << 20) | ((uint64_t)fa.slab << 8) | ((uint64_t)fa.group << 3) |
                       ((uint64_t)grad << 2) | ((uint64_t)kahan << 1) | (uint64_t)c->bf16;
  auto oc = c->occupancy.find(key);
  int bps = 0;
  if (oc == c->occupancy.end()) {
    cudaError_t oe = fused_blocks_per_sm(fa, grad, kahan, c->bf16, &bps);
    if (oe != cudaSuccess) return cuda_fail(c, oe, "occupancy query");
    if (bps < 1) return fail(c, GWC_E_UNSUPPORTED, "the fused kernel does not fit on an SM at this geometry");
    c->occupancy[key] = bps;
  } else {
    bps = oc->second;
  }
  const long long grid = std::max(1LL, std::min(units, (long long)c->n_sms * bps));
  cudaError_t e = launch_fused(fa, grad, kahan, c->bf16, (int)grid, s);
  if (e != cudaSuccess) return cuda_fail(c, e, "sample kernel launch");
  return GWC_OK;
}

gwc_status run_fused(gwc_ctx* c, int32_t K, const double* d_lambda, double* lnL_event,
                     double* neff_event, double* ln_xi, double* neff_sel, double* lnL_total,
                     int32_t* flags, double* grad_total, bool grad, cudaStream_t s,
                     double* sum_events = nullptr, double* grad_events = nullptr,
                     double* grad_ln_xi = nullptr) {
  cudaError_t pe = prof_mark(c, 0, s);
  if (pe != cudaSuccess) return cuda_fail(c, pe, "profile event");
  gwc_status st = run_prologue(c, K, d_lambda, grad, s, c->counter);
  if (st != GWC_OK) return st;
  if ((pe = prof_mark(c, 1, s)) != cudaSuccess) return cuda_fail(c, pe, "profile event");
  st = launch_fused_items(c, K, grad, c->sched, c->n_items, c->partials, c->n_items, 0, s);
  if (st != GWC_OK) return st;
  cudaError_t e;
  if ((e = prof_mark(c, 2, s)) != cudaSuccess) return cuda_fail(c, e, "profile event");
  st = run_merge(c, K, 1, grad, lnL_event, neff_event, ln_xi, neff_sel, lnL_total, flags,
                 grad_total, s, sum_events, grad_events, grad_ln_xi);
  if (st != GWC_OK) return st;
  if ((e = prof_mark(c, 3, s)) != cudaSuccess) return cuda_fail(c, e, "profile event");
  return GWC_OK;
}

// Switch the context to another chunk size: re-split the work items and upload them
// (growing the item and partial buffers when needed).  The caller has synchronised.
gwc_status set_chunk(gwc_ctx* c, int chunk) {
  if (chunk == c->opt.chunk) return GWC_OK;
  ItemLayout lay;
  if (!make_items(c->h_offsets.data(), c->n_events, c->n_samples, c->n_inj, chunk, lay))
    return fail(c, GWC_E_INVALID, "too many work items");
  const int64_t n = (int64_t)lay.items.size();
  if (n > c->items_cap) {
    Item* it = nullptr;
    int32_t* sc = nullptr;
    float* pa = nullptr;
    cudaError_t e = cudaMalloc(reinterpret_cast<void**>(&it), sizeof(Item) * (size_t)n);
    if (e == cudaSuccess) e = cudaMalloc(reinterpret_cast<void**>(&sc), sizeof(int32_t) * (size_t)n);
    if (e == cudaSuccess)
      e = cudaMalloc(reinterpret_cast<void**>(&pa), sizeof(float) * (size_t)c->opt.max_K * (size_t)n * PSTRIDE);
    if (e != cudaSuccess) {
      if (it) cudaFree(it);
      if (sc) cudaFree(sc);
      cudaGetLastError();
      return fail(c, e == cudaErrorMemoryAllocation ? GWC_E_NOMEM : GWC_E_CUDA,
                  std::string("work-item buffers: ") + cudaGetErrorString(e));
    }
    cudaFree(c->items);
    cudaFree(c->sched);
    cudaFree(c->partials);
    c->device_bytes += (n - c->items_cap) * (int64_t)(sizeof(Item) + sizeof(int32_t) +
                                                      sizeof(float) * (size_t)c->opt.max_K * PSTRIDE);
    c->items = it;
    c->sched = sc;
    c->partials = pa;
    c->items_cap = n;
  }
  cudaError_t e = cudaMemcpy(c->items, lay.items.data(), sizeof(Item) * (size_t)n, cudaMemcpyHostToDevice);
  if (e == cudaSuccess)
    e = cudaMemcpy(c->sched, lay.sched.data(), sizeof(int32_t) * (size_t)n, cudaMemcpyHostToDevice);
  if (e == cudaSuccess)
    e = cudaMemcpy(c->ev_item0, lay.ev_item0.data(), sizeof(int32_t) * lay.ev_item0.size(), cudaMemcpyHostToDevice);
  if (e == cudaSuccess && c->sample_item)
    e = cudaMemcpy(c->sample_item, lay.sample_item.data(), sizeof(int32_t) * lay.sample_item.size(),
                   cudaMemcpyHostToDevice);
  if (e != cudaSuccess) return cuda_fail(c, e, "work-item upload");
  c->n_items = (int32_t)n;
  c->inj_item0 = lay.inj_item0;
  c->h_sample_item = std::move(lay.sample_item);
  c->opt.chunk = chunk;
  // the KDE form's injection schedule and partial buffer follow the item layout
  if (c->kde_sched_inj) { cudaFree(c->kde_sched_inj); c->kde_sched_inj = nullptr; }
  if (c->kde_partials) { cudaFree(c->kde_partials); c->kde_partials = nullptr; }
  return GWC_OK;
}

// Device resources of the KDE form, made on first use (and the LOS grid table again when
// the grid size changes).
gwc_status kde_prepare(gwc_ctx* c, int G, cudaStream_t s) {
  auto oom = [&](cudaError_t e, const char* what) {
    cudaGetLastError();
    return fail(c, e == cudaErrorMemoryAllocation ? GWC_E_NOMEM : GWC_E_CUDA,
                std::string(what) + ": " + cudaGetErrorString(e));
  };
  cudaError_t e = cudaSuccess;
  const size_t ng = c->h_groups.size();
  if (!c->kde_groups && ng > 0) {
    e = dalloc(c, &c->kde_groups, ng);
    if (e == cudaSuccess) e = cudaMemcpy(c->kde_groups, c->h_groups.data(), sizeof(KdeGroup) * ng, cudaMemcpyHostToDevice);
    if (e != cudaSuccess) return oom(e, "KDE groups");
  }
  if (!c->kde_ev_group0) {
    e = dalloc(c, &c->kde_ev_group0, c->h_ev_group0.size());
    if (e == cudaSuccess)
      e = cudaMemcpy(c->kde_ev_group0, c->h_ev_group0.data(), sizeof(int32_t) * c->h_ev_group0.size(),
                     cudaMemcpyHostToDevice);
    if (e != cudaSuccess) return oom(e, "KDE group offsets");
  }
  if (!c->kde_sched_inj) {
    ItemLayout lay;
    if (!make_items(c->h_offsets.data(), c->n_events, c->n_samples, c->n_inj, c->opt.chunk, lay))
      return fail(c, GWC_E_INVALID, "too many work items");
    std::vector<int32_t> si;
    for (int32_t q : lay.sched)
      if (q >= lay.inj_item0) si.push_back(q);
    e = dalloc(c, &c->kde_sched_inj, std::max<size_t>(si.size(), 1));
    if (e == cudaSuccess && !si.empty())
      e = cudaMemcpy(c->kde_sched_inj, si.data(), sizeof(int32_t) * si.size(), cudaMemcpyHostToDevice);
    if (e != cudaSuccess) return oom(e, "KDE injection schedule");
  }
  if (!c->kde_partials) {
    c->kde_stride = (int64_t)ng + c->n_items;
    e = dalloc(c, &c->kde_partials, (size_t)c->opt.max_K * (size_t)c->kde_stride * PSTRIDE);
    if (e != cudaSuccess) return oom(e, "KDE partials");
  }
  if (!c->kde_lm && c->n_samples > 0) {
    e = dalloc(c, &c->kde_lm, (size_t)c->n_samples);
    if (e != cudaSuccess) return oom(e, "KDE log2 masses");
    e = launch_log2_masses(c->smp, c->n_samples, c->kde_lm, s);
    if (e != cudaSuccess) return cuda_fail(c, e, "KDE log2 masses");
  }
  if (c->kde_G != G) {
    if (c->kde_pgrid) { cudaFree(c->kde_pgrid); c->kde_pgrid = nullptr; c->kde_G = 0; }
    e = dalloc(c, &c->kde_pgrid, (size_t)c->n_pix * kde_row(G));
    if (e != cudaSuccess) return oom(e, "KDE grid table");
    e = launch_los_grid(static_cast<const float*>(c->los), c->n_pix, c->n_z, c->z_max, G, c->kde_pgrid, s);
    if (e != cudaSuccess) return cuda_fail(c, e, "KDE grid table");
    c->kde_G = G;
  }
  return GWC_OK;
}

}  // namespace

extern "C" {

void gwc_default_options(gwc_options* o) {
  if (!o) return;
  o->neff_min_event = 2.0;
  o->neff_min_sel = 0.0;
  o->accum = 0;
  o->los_dtype = GWC_LOS_F32;
  o->n_x_table = 512;
  o->max_K = 256;
  o->chunk = 2048;
  o->lambda_tile = 0;
  o->lambda_group = 0;
  o->cap_per_pixel = 0;
  o->cap_seed = 0;
  o->mass_model = GWC_MASS_PLP;
}

gwc_status gwc_create(const gwc_events* ev, const gwc_los* los, const gwc_injections* inj,
                      const gwc_options* opts, gwc_ctx** out) {
  if (!out) return fail(nullptr, GWC_E_INVALID, "out is NULL");
  *out = nullptr;
  if (!ev || !los || !inj) return fail(nullptr, GWC_E_INVALID, "NULL events, LOS or injections");
  gwc_options o;
  gwc_default_options(&o);
  if (opts) o = *opts;
  if (o.max_K < 1 || o.max_K > 65535) return fail(nullptr, GWC_E_INVALID, "max_K must be in [1, 65535]");
  if (o.n_x_table < 16 || o.n_x_table > 4096 || o.n_x_table % 4 != 0)
    return fail(nullptr, GWC_E_INVALID, "n_x_table must be a multiple of 4 in [16, 4096]");
  if (o.chunk < 64 || o.chunk > 4096) return fail(nullptr, GWC_E_INVALID, "chunk must be in [64, 4096]");
  if (o.accum != 0 && o.accum != 1) return fail(nullptr, GWC_E_INVALID, "accum must be 0 or 1");
  if (o.los_dtype != GWC_LOS_F32 && o.los_dtype != GWC_LOS_BF16) return fail(nullptr, GWC_E_INVALID, "bad los_dtype");
  if (o.lambda_group != 0 && o.lambda_group != 1 && o.lambda_group != 2 && o.lambda_group != 4 &&
      o.lambda_group != 8)
    return fail(nullptr, GWC_E_INVALID, "lambda_group must be 0 (default), 1, 2, 4 or 8");
  if (o.lambda_tile < 0 || o.lambda_tile > MAX_SLAB)
    return fail(nullptr, GWC_E_INVALID, "lambda_tile must be in [0, " + std::to_string(MAX_SLAB) + "]");
  if (!(o.neff_min_event >= 0.0) || !(o.neff_min_sel >= 0.0)) return fail(nullptr, GWC_E_INVALID, "N_eff thresholds must be >= 0");
  if (o.cap_per_pixel < 0) return fail(nullptr, GWC_E_INVALID, "cap_per_pixel must be >= 0");
  if (o.mass_model != GWC_MASS_PLP && o.mass_model != GWC_MASS_MULTIPEAK)
    return fail(nullptr, GWC_E_INVALID, "mass_model must be GWC_MASS_PLP or GWC_MASS_MULTIPEAK");

  // ---- validate the events
  const int32_t ne = ev->n_events;
  if (ne < 0) return fail(nullptr, GWC_E_INVALID, "n_events < 0");
  if (!ev->offsets) return fail(nullptr, GWC_E_INVALID, "offsets is NULL");
  if (ev->offsets[0] != 0) return fail(nullptr, GWC_E_INVALID, "offsets[0] must be 0");
  for (int32_t e = 0; e < ne; ++e)
    if (ev->offsets[e + 1] <= ev->offsets[e])
      return fail(nullptr, GWC_E_INVALID, "offsets must be strictly increasing (event " + std::to_string(e) + ")");
  int64_t ns = ev->offsets[ne];
  if (ns > 0 && (!ev->m1_det || !ev->m2_det || !ev->dl_mpc || !ev->ln_pe_prior || !ev->pix))
    return fail(nullptr, GWC_E_INVALID, "NULL sample array");
  if (!finite_all(ev->m1_det, ns) || !finite_all(ev->m2_det, ns) || !finite_all(ev->dl_mpc, ns) ||
      !finite_all(ev->ln_pe_prior, ns))
    return fail(nullptr, GWC_E_INVALID, "non-finite sample value");
  // ---- LOS
  if (los->n_pix < 1 || los->n_z < 2 || los->n_z > (1 << 24)) return fail(nullptr, GWC_E_INVALID, "need n_pix >= 1 and 2 <= n_z <= 2^24");
  if (!(los->z_max > 0.0) || !std::isfinite(los->z_max)) return fail(nullptr, GWC_E_INVALID, "z_max must be finite and > 0");
  if (los->dtype != GWC_LOS_F32 && los->dtype != GWC_LOS_BF16) return fail(nullptr, GWC_E_INVALID, "bad LOS dtype");
  if (!los->p_z) return fail(nullptr, GWC_E_INVALID, "LOS table is NULL");
  for (int64_t k = 0; k < ns; ++k)
    if (ev->pix[k] < 0 || ev->pix[k] >= los->n_pix)
      return fail(nullptr, GWC_E_INVALID, "pixel id out of range at sample " + std::to_string(k));
  // ---- per-pixel cap (the paper's memory option): in each (event, pixel) group larger
  //      than the cap keep the cap samples with the smallest key, the (k+1)-th output of
  //      SplitMix64 started at cap_seed for input sample k
  gwc_events evc{};
  std::vector<float> cm1, cm2, cdl, clp;
  std::vector<int32_t> cpx;
  std::vector<int64_t> coff;
  if (o.cap_per_pixel > 0) {
    auto key = [&](int64_t k) {
      uint64_t z = o.cap_seed + (uint64_t)(k + 1) * 0x9e3779b97f4a7c15ull;
      z = (z ^ (z >> 30)) * 0xbf58476d1ce4e5b9ull;
      z = (z ^ (z >> 27)) * 0x94d049bb133111ebull;
      return z ^ (z >> 31);
    };
    coff.assign((size_t)ne + 1, 0);
    std::vector<int64_t> idx, kept;
    for (int32_t e = 0; e < ne; ++e) {
      idx.clear();
      for (int64_t k = ev->offsets[e]; k < ev->offsets[e + 1]; ++k) idx.push_back(k);
      std::stable_sort(idx.begin(), idx.end(), [&](int64_t a, int64_t b) { return ev->pix[a] < ev->pix[b]; });
      kept.clear();
      for (size_t a = 0; a < idx.size();) {
        size_t b = a;
        while (b < idx.size() && ev->pix[idx[b]] == ev->pix[idx[a]]) ++b;
        if ((int64_t)(b - a) > o.cap_per_pixel) {
          std::vector<int64_t> run(idx.begin() + a, idx.begin() + b);
          std::nth_element(run.begin(), run.begin() + o.cap_per_pixel, run.end(),
                           [&](int64_t x, int64_t y) { return key(x) < key(y); });
          kept.insert(kept.end(), run.begin(), run.begin() + o.cap_per_pixel);
        } else {
          kept.insert(kept.end(), idx.begin() + a, idx.begin() + b);
        }
        a = b;
      }
      std::sort(kept.begin(), kept.end());   // input order within the event
      for (int64_t k : kept) {
        cm1.push_back(ev->m1_det[k]);
        cm2.push_back(ev->m2_det[k]);
        cdl.push_back(ev->dl_mpc[k]);
        clp.push_back(ev->ln_pe_prior[k]);
        cpx.push_back(ev->pix[k]);
      }
      coff[(size_t)e + 1] = (int64_t)cm1.size();
    }
    evc.n_events = ne;
    evc.offsets = coff.data();
    evc.m1_det = cm1.data();
    evc.m2_det = cm2.data();
    evc.dl_mpc = cdl.data();
    evc.ln_pe_prior = clp.data();
    evc.pix = cpx.data();
    ev = &evc;
    ns = coff[(size_t)ne];
  }
  const int64_t nlos = (int64_t)los->n_pix * los->n_z;
  std::vector<float> los_f((size_t)nlos);
  if (los->dtype == GWC_LOS_F32) {
    std::memcpy(los_f.data(), los->p_z, sizeof(float) * (size_t)nlos);
  } else {
    const uint16_t* h = static_cast<const uint16_t*>(los->p_z);
    for (int64_t i = 0; i < nlos; ++i) los_f[(size_t)i] = from_bf16(h[i]);
  }
  for (int64_t i = 0; i < nlos; ++i)
    if (!std::isfinite(los_f[(size_t)i]) || los_f[(size_t)i] < 0.f)
      return fail(nullptr, GWC_E_INVALID, "LOS values must be finite and >= 0");
  // ---- injections
  if (inj->n_found < 1) return fail(nullptr, GWC_E_INVALID, "need at least one injection");
  if (!(inj->n_draw >= (double)inj->n_found) || !std::isfinite(inj->n_draw))
    return fail(nullptr, GWC_E_INVALID, "n_draw must be finite and >= n_found");
  if (!inj->m1_det || !inj->m2_det || !inj->dl_mpc || !inj->ln_p_draw) return fail(nullptr, GWC_E_INVALID, "NULL injection array");
  const int64_t ni = inj->n_found;
  if (!finite_all(inj->m1_det, ni) || !finite_all(inj->m2_det, ni) || !finite_all(inj->dl_mpc, ni) ||
      !finite_all(inj->ln_p_draw, ni))
    return fail(nullptr, GWC_E_INVALID, "non-finite injection value");

  int dev = 0;
  cudaError_t ce = cudaGetDevice(&dev);
  if (ce != cudaSuccess) return fail(nullptr, GWC_E_UNSUPPORTED, std::string("no CUDA device: ") + cudaGetErrorString(ce));

  gwc_ctx* c = new (std::nothrow) gwc_ctx();
  if (!c) return fail(nullptr, GWC_E_NOMEM, "host allocation failed");
  c->device = dev;
  c->opt = o;
  c->n_events = ne;
  c->n_samples = ns;
  c->n_inj = ni;
  c->n_draw = inj->n_draw;
  c->n_pix = los->n_pix;
  c->n_z = los->n_z;
  c->z_max = los->z_max;
  c->bf16 = o.los_dtype == GWC_LOS_BF16;
  c->mp = o.mass_model == GWC_MASS_MULTIPEAK;
  c->np = n_params(c->mp);
  c->tstride = (table_floats(o.n_x_table) + 3) & ~3;

  // ---- host layout: samples sorted by pixel inside each event, work items
  std::vector<float4> h_smp((size_t)ns);
  std::vector<int32_t> h_pix((size_t)ns);
  {
    std::vector<int64_t> idx;
    for (int32_t e = 0; e < ne; ++e) {
      const int64_t a = ev->offsets[e], b = ev->offsets[e + 1];
      idx.resize((size_t)(b - a));
      for (int64_t k = a; k < b; ++k) idx[(size_t)(k - a)] = k;
      // by pixel (few LOS rows per chunk), then by d_L: a warp's 32 lanes then read
      // neighbouring nodes of the inversion table and neighbouring cells of the LOS row
      std::stable_sort(idx.begin(), idx.end(), [&](int64_t x, int64_t y) {
        return ev->pix[x] < ev->pix[y] || (ev->pix[x] == ev->pix[y] && ev->dl_mpc[x] < ev->dl_mpc[y]);
      });

      for (int64_t q = 0; q < b - a; ++q) {
        const int64_t k = idx[(size_t)q];
        h_smp[(size_t)(a + q)] = make_float4(ev->m1_det[k], ev->m2_det[k], ev->dl_mpc[k], ev->ln_pe_prior[k]);
        h_pix[(size_t)(a + q)] = ev->pix[k];
      }
    }
  }
  // (event, pixel) groups of the sorted samples, for the KDE form
  c->h_ev_group0.assign((size_t)ne + 1, 0);
  for (int32_t e = 0; e < ne; ++e) {
    c->h_ev_group0[(size_t)e] = (int32_t)c->h_groups.size();
    for (int64_t q = ev->offsets[e]; q < ev->offsets[e + 1];) {
      int64_t r = q;
      while (r < ev->offsets[e + 1] && h_pix[(size_t)r] == h_pix[(size_t)q]) ++r;
      c->h_groups.push_back(KdeGroup{q, (int32_t)(r - q), h_pix[(size_t)q]});
      q = r;
    }
  }
  c->h_ev_group0[(size_t)ne] = (int32_t)c->h_groups.size();
  // injections by d_L, for the same reason (their sum does not depend on the order), then
  // each block of INJ_BLOCK by m1_det: a block spans so little d_L that z is almost the
  // same for all of it, so the injections above m_max (1 + z) -- often 40% of a broad
  // injection set -- gather into whole warps that leave the loop early
  std::vector<float4> h_inj((size_t)ni);
  {
    std::vector<int64_t> idx((size_t)ni);
    for (int64_t k = 0; k < ni; ++k) idx[(size_t)k] = k;
    std::stable_sort(idx.begin(), idx.end(),
                     [&](int64_t x, int64_t y) { return inj->dl_mpc[x] < inj->dl_mpc[y]; });
    for (size_t q0 = 0; q0 < idx.size(); q0 += INJ_BLOCK)
      std::stable_sort(idx.begin() + q0, idx.begin() + std::min(idx.size(), q0 + INJ_BLOCK),
                       [&](int64_t x, int64_t y) { return inj->m1_det[x] < inj->m1_det[y]; });
    for (int64_t q = 0; q < ni; ++q) {
      const int64_t k = idx[(size_t)q];
      h_inj[(size_t)q] = make_float4(inj->m1_det[k], inj->m2_det[k], inj->dl_mpc[k], inj->ln_p_draw[k]);
    }
  }
  std::vector<double> ln_ev_n((size_t)std::max(ne, 1));
  for (int32_t e = 0; e < ne; ++e) ln_ev_n[(size_t)e] = std::log((double)(ev->offsets[e + 1] - ev->offsets[e]));
  c->h_offsets.assign(ev->offsets, ev->offsets + (size_t)ne + 1);
  ItemLayout lay;
  if (!make_items(ev->offsets, ne, ns, ni, o.chunk, lay)) {
    delete c;
    return fail(nullptr, GWC_E_INVALID, "too many work items");
  }
  c->n_items = (int32_t)lay.items.size();
  c->items_cap = c->n_items;
  c->inj_item0 = lay.inj_item0;
  c->h_sample_item = std::move(lay.sample_item);
  const std::vector<Item>& items = lay.items;
  const std::vector<int32_t>& sched = lay.sched;
  const std::vector<int32_t>& ev_item0 = lay.ev_item0;
  // pixel mean of the LOS rows (the selection term's redshift prior)
  std::vector<double> pbar((size_t)c->n_z, 0.0);
  for (int32_t p = 0; p < c->n_pix; ++p)
    for (int32_t j = 0; j < c->n_z; ++j) pbar[(size_t)j] += (double)los_f[(size_t)p * c->n_z + j];
  std::vector<float> pbar32((size_t)c->n_z);
  for (int32_t j = 0; j < c->n_z; ++j) {
    pbar[(size_t)j] /= (double)c->n_pix;
    pbar32[(size_t)j] = (float)pbar[(size_t)j];
  }

  // ---- device memory
  const int kcap = o.max_K;
  cudaError_t e = cudaSuccess;
  auto chk = [&](cudaError_t r) { if (e == cudaSuccess) e = r; };
  chk(dalloc(c, &c->smp, (size_t)ns));
  chk(dalloc(c, &c->pix, (size_t)ns));
  chk(dalloc(c, &c->inj, (size_t)ni));
  if (c->bf16) {
    uint16_t* p = nullptr;
    chk(dalloc(c, &p, (size_t)nlos));
    c->los = p;
  } else {
    float* p = nullptr;
    chk(dalloc(c, &p, (size_t)nlos));
    c->los = p;
  }
  chk(dalloc(c, &c->pbar32, (size_t)c->n_z));
  chk(dalloc(c, &c->pbar64, (size_t)c->n_z));
  chk(dalloc(c, &c->items, items.size()));
  chk(dalloc(c, &c->sched, sched.size()));
  chk(dalloc(c, &c->ev_item0, ev_item0.size()));
  chk(dalloc(c, &c->ln_ev_n, ln_ev_n.size()));
  chk(dalloc(c, &c->lf, (size_t)o.max_K));
  chk(dalloc(c, &c->ld, (size_t)o.max_K));
  chk(dalloc(c, &c->tables, (size_t)o.max_K * c->tstride));
  chk(dalloc(c, &c->partials, (size_t)kcap * c->n_items * PSTRIDE));
  chk(dalloc(c, &c->counter, 1));
  chk(dalloc(c, &c->order, (size_t)o.max_K));
  chk(cudaDeviceGetAttribute(&c->n_sms, cudaDevAttrMultiProcessorCount, c->device));
  chk(dalloc(c, &c->d_lam, (size_t)o.max_K * NP_MAX));
  chk(dalloc(c, &c->d_out, (size_t)o.max_K * (2 * (size_t)std::max(ne, 1) + 3 + NP_MAX)));
  chk(dalloc(c, &c->d_flags, (size_t)o.max_K));
  if (e == cudaSuccess) e = cudaMallocHost(reinterpret_cast<void**>(&c->h_lam), sizeof(double) * o.max_K * NP_MAX);
  if (e == cudaSuccess) e = cudaMallocHost(reinterpret_cast<void**>(&c->h_out), sizeof(double) * o.max_K * (1 + NP_MAX));
  if (e == cudaSuccess) e = cudaMallocHost(reinterpret_cast<void**>(&c->h_flags), sizeof(int32_t) * o.max_K);
  if (e != cudaSuccess) {
    const bool oom = e == cudaErrorMemoryAllocation;
    std::string msg = std::string("allocation failed: ") + cudaGetErrorString(e);
    cudaGetLastError();
    free_all(c);
    delete c;
    return fail(nullptr, oom ? GWC_E_NOMEM : GWC_E_CUDA, msg);
  }
  chk(cudaMemcpy(c->smp, h_smp.data(), sizeof(float4) * (size_t)ns, cudaMemcpyHostToDevice));
  chk(cudaMemcpy(c->pix, h_pix.data(), sizeof(int32_t) * (size_t)ns, cudaMemcpyHostToDevice));
  chk(cudaMemcpy(c->inj, h_inj.data(), sizeof(float4) * (size_t)ni, cudaMemcpyHostToDevice));
  if (c->bf16) {
    std::vector<uint16_t> hb((size_t)nlos);
    for (int64_t i = 0; i < nlos; ++i) hb[(size_t)i] = to_bf16(los_f[(size_t)i]);
    chk(cudaMemcpy(c->los, hb.data(), sizeof(uint16_t) * (size_t)nlos, cudaMemcpyHostToDevice));
  } else {
    chk(cudaMemcpy(c->los, los_f.data(), sizeof(float) * (size_t)nlos, cudaMemcpyHostToDevice));
  }
  chk(cudaMemcpy(c->pbar32, pbar32.data(), sizeof(float) * pbar32.size(), cudaMemcpyHostToDevice));
  chk(cudaMemcpy(c->pbar64, pbar.data(), sizeof(double) * pbar.size(), cudaMemcpyHostToDevice));
  chk(cudaMemcpy(c->items, items.data(), sizeof(Item) * items.size(), cudaMemcpyHostToDevice));
  chk(cudaMemcpy(c->sched, sched.data(), sizeof(int32_t) * sched.size(), cudaMemcpyHostToDevice));
  chk(cudaMemcpy(c->ev_item0, ev_item0.data(), sizeof(int32_t) * ev_item0.size(), cudaMemcpyHostToDevice));
  chk(cudaMemcpy(c->ln_ev_n, ln_ev_n.data(), sizeof(double) * ln_ev_n.size(), cudaMemcpyHostToDevice));
  chk(ensure_prologue_ready());
  if (e != cudaSuccess) {
    std::string msg = std::string("device upload failed: ") + cudaGetErrorString(e);
    free_all(c);
    delete c;
    return fail(nullptr, GWC_E_CUDA, msg);
  }
  {
    std::lock_guard<std::mutex> g(g_mu);
    static uint64_t next_serial = 0;
    c->serial = ++next_serial;
    g_live.insert(c);
  }
  *out = c;
  return GWC_OK;
}

gwc_status gwc_loglik(gwc_ctx* c, int32_t K, const double* d_lambda, double* d_lnL_event,
                      double* d_neff_event, double* d_ln_xi, double* d_neff_sel,
                      double* d_lnL_total, int32_t* d_flags, void* stream) {
  gwc_status st = check_call(c, K, d_lambda, d_lnL_event, d_neff_event, d_ln_xi, d_neff_sel,
                             d_lnL_total, d_flags);
  if (st != GWC_OK) return st;
  return run_fused(c, K, d_lambda, d_lnL_event, d_neff_event, d_ln_xi, d_neff_sel, d_lnL_total,
                   d_flags, nullptr, false, static_cast<cudaStream_t>(stream));
}

gwc_status gwc_loglik_grad(gwc_ctx* c, int32_t K, const double* d_lambda, double* d_lnL_event,
                           double* d_neff_event, double* d_ln_xi, double* d_neff_sel,
                           double* d_lnL_total, int32_t* d_flags, double* d_grad_total,
                           void* stream) {
  gwc_status st = check_call(c, K, d_lambda, d_lnL_event, d_neff_event, d_ln_xi, d_neff_sel,
                             d_lnL_total, d_flags);
  if (st != GWC_OK) return st;
  if (!d_grad_total) return fail(c, GWC_E_INVALID, "d_grad_total is NULL");
  return run_fused(c, K, d_lambda, d_lnL_event, d_neff_event, d_ln_xi, d_neff_sel, d_lnL_total,
                   d_flags, d_grad_total, true, static_cast<cudaStream_t>(stream));
}

void gwc_default_kde_options(gwc_kde_options* o) {
  if (!o) return;
  o->bw_rule = GWC_BW_SCOTT;
  o->n_grid = 256;
  o->neff_min_pixel = 2.0;
}

namespace {
gwc_status kde_options_check(gwc_ctx* c, const gwc_kde_options* kopt, gwc_kde_options* ko) {
  gwc_default_kde_options(ko);
  if (kopt) *ko = *kopt;
  if (ko->bw_rule < GWC_BW_SCOTT || ko->bw_rule > GWC_BW_BIWEIGHT)
    return fail(c, GWC_E_INVALID, "bw_rule must be GWC_BW_SCOTT, GWC_BW_SILVERMAN or GWC_BW_BIWEIGHT");
  if (ko->n_grid < 2 || ko->n_grid > 65536) return fail(c, GWC_E_INVALID, "n_grid must be in [2, 65536]");
  if (!(ko->neff_min_pixel >= 0.0)) return fail(c, GWC_E_INVALID, "neff_min_pixel must be >= 0");
  if (c->bf16) return fail(c, GWC_E_UNSUPPORTED, "the KDE form needs the LOS table stored as FP32");
  return GWC_OK;
}

KdeArgs kde_args(gwc_ctx* c, const gwc_kde_options& ko, int32_t K) {
  KdeArgs ka;
  ka.smp = c->smp;
  ka.lm = c->kde_lm;
  ka.groups = c->kde_groups;
  ka.n_groups = (int)c->h_groups.size();
  ka.pgrid = c->kde_pgrid;
  ka.G = ko.n_grid;
  ka.dzg = (float)(c->z_max / (ko.n_grid - 1));
  ka.rule = ko.bw_rule;
  ka.neff_min = (float)ko.neff_min_pixel;
  ka.K = K;
  ka.nx = c->opt.n_x_table;
  ka.nz = c->n_z;
  ka.lf = c->lf;
  ka.tables = c->tables;
  ka.tstride = c->tstride;
  ka.partials = c->kde_partials;
  ka.stride = (int)c->kde_stride;
  ka.mp = c->mp ? 1 : 0;
  return ka;
}
}  // namespace

gwc_status gwc_loglik_kde(gwc_ctx* c, int32_t K, const double* d_lambda, const gwc_kde_options* kopt,
                          double* d_lnL_event, double* d_neff_event, double* d_ln_xi,
                          double* d_neff_sel, double* d_lnL_total, int32_t* d_flags, void* stream) {
  gwc_status st = check_call(c, K, d_lambda, d_lnL_event, d_neff_event, d_ln_xi, d_neff_sel,
                             d_lnL_total, d_flags);
  if (st != GWC_OK) return st;
  gwc_kde_options ko;
  if ((st = kde_options_check(c, kopt, &ko)) != GWC_OK) return st;
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  st = kde_prepare(c, ko.n_grid, s);
  if (st != GWC_OK) return st;
  cudaError_t pe = prof_mark(c, 0, s);
  if (pe != cudaSuccess) return cuda_fail(c, pe, "profile event");
  st = run_prologue(c, K, d_lambda, false, s, c->counter);
  if (st != GWC_OK) return st;
  const int64_t ng = (int64_t)c->h_groups.size();
  // the selection term: the Monte-Carlo sum over the injections only (profiled with the
  // prologue, so that the second stage is the KDE kernel alone)
  st = launch_fused_items(c, K, false, c->kde_sched_inj, c->n_items - c->inj_item0, c->kde_partials,
                          c->kde_stride, ng, s);
  if (st != GWC_OK) return st;
  if ((pe = prof_mark(c, 1, s)) != cudaSuccess) return cuda_fail(c, pe, "profile event");
  const KdeArgs ka = kde_args(c, ko, K);
  cudaError_t e = launch_kde(ka, s);
  if (e != cudaSuccess) return cuda_fail(c, e, "KDE launch");
  if ((e = prof_mark(c, 2, s)) != cudaSuccess) return cuda_fail(c, e, "profile event");
  MergeArgs ma;
  ma.partials = c->kde_partials;
  ma.n_items = (int)c->kde_stride;
  ma.P = 1;
  ma.ev_item0 = c->kde_ev_group0;
  ma.n_events = c->n_events;
  ma.inj_item0 = (int)(ng + c->inj_item0);
  ma.ln_ev_n = c->ln_ev_n;
  ma.ln_n_draw = std::log(c->n_draw);
  ma.ld = c->ld;
  ma.neff_min_event = 0.0;   // the per-pixel cut replaces the per-event one
  ma.neff_min_sel = c->opt.neff_min_sel;
  ma.lnL_event = d_lnL_event;
  ma.neff_event = d_neff_event;
  ma.ln_xi = d_ln_xi;
  ma.neff_sel = d_neff_sel;
  ma.lnL_total = d_lnL_total;
  ma.flags = d_flags;
  ma.grad_total = nullptr;
  e = launch_merge(ma, K, false, s);
  if (e != cudaSuccess) return cuda_fail(c, e, "merge launch");
  if ((e = prof_mark(c, 3, s)) != cudaSuccess) return cuda_fail(c, e, "profile event");
  return GWC_OK;
}

gwc_status gwc_loglik_parts(gwc_ctx* c, int32_t K, const double* d_lambda, double* d_lnL_event,
                            double* d_neff_event, double* d_ln_xi, double* d_neff_sel,
                            double* d_sum_events, int32_t* d_flags, double* d_grad_events,
                            double* d_grad_ln_xi, void* stream) {
  if (!d_sum_events) return fail(c, GWC_E_INVALID, "d_sum_events is NULL");
  if ((d_grad_events == nullptr) != (d_grad_ln_xi == nullptr))
    return fail(c, GWC_E_INVALID, "give both gradient parts or neither");
  // check_call requires a non-NULL total pointer; d_sum_events stands in for it
  gwc_status st = check_call(c, K, d_lambda, d_lnL_event, d_neff_event, d_ln_xi, d_neff_sel,
                             d_sum_events, d_flags);
  if (st != GWC_OK) return st;
  const bool grad = d_grad_events != nullptr;
  return run_fused(c, K, d_lambda, d_lnL_event, d_neff_event, d_ln_xi, d_neff_sel, nullptr, d_flags,
                   nullptr, grad, static_cast<cudaStream_t>(stream), d_sum_events, d_grad_events,
                   d_grad_ln_xi);
}

gwc_status gwc_loglik_plain(gwc_ctx* c, int32_t K, const double* d_lambda, double* d_lnL_event,
                            double* d_neff_event, double* d_ln_xi, double* d_neff_sel,
                            double* d_lnL_total, int32_t* d_flags, double* d_grad_total,
                            void* stream) {
  gwc_status st = check_call(c, K, d_lambda, d_lnL_event, d_neff_event, d_ln_xi, d_neff_sel,
                             d_lnL_total, d_flags);
  if (st != GWC_OK) return st;
  if (c->mp) return fail(c, GWC_E_UNSUPPORTED, "the plain path evaluates the power law + peak model only");
  const bool grad = d_grad_total != nullptr;
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  const long long ntot = c->n_samples + c->n_inj;
  if (!c->plain_lw) {   // scratch of the baseline path, allocated on its first use
    cudaError_t e = dalloc(c, &c->plain_lw, (size_t)ntot);
    if (e == cudaSuccess) e = dalloc(c, &c->plain_tg, (size_t)ntot * NP);
    if (e == cudaSuccess) e = dalloc(c, &c->sample_item, (size_t)ntot);
    if (e == cudaSuccess)
      e = cudaMemcpy(c->sample_item, c->h_sample_item.data(), sizeof(int32_t) * (size_t)ntot,
                     cudaMemcpyHostToDevice);
    if (e != cudaSuccess) {
      const bool oom = e == cudaErrorMemoryAllocation;
      cudaGetLastError();
      if (c->plain_lw) cudaFree(c->plain_lw);
      if (c->plain_tg) cudaFree(c->plain_tg);
      if (c->sample_item) cudaFree(c->sample_item);
      c->plain_lw = nullptr;
      c->plain_tg = nullptr;
      c->sample_item = nullptr;
      return fail(c, oom ? GWC_E_NOMEM : GWC_E_CUDA, std::string("plain-path scratch: ") + cudaGetErrorString(e));
    }
  }
  cudaError_t pe = prof_mark(c, 0, s);
  if (pe != cudaSuccess) return cuda_fail(c, pe, "profile event");
  st = run_prologue(c, K, d_lambda, grad, s);
  if (st != GWC_OK) return st;
  if ((pe = prof_mark(c, 1, s)) != cudaSuccess) return cuda_fail(c, pe, "profile event");
  PlainArgs pa;
  pa.smp = c->smp;
  pa.pix = c->pix;
  pa.inj = c->inj;
  pa.los = c->los;
  pa.pbar32 = c->pbar32;
  pa.nz = c->n_z;
  pa.nx = c->opt.n_x_table;
  pa.n_samples = c->n_samples;
  pa.n_total = ntot;
  pa.items = c->items;
  pa.sample_item = c->sample_item;
  pa.n_items = c->n_items;
  pa.lf = c->lf;
  pa.tables = c->tables;
  pa.tstride = c->tstride;
  pa.lw = c->plain_lw;
  pa.tg = c->plain_tg;
  pa.partials = c->partials;
  for (int k = 0; k < K; ++k) {
    pa.k = k;
    cudaError_t e = launch_plain_sample(pa, false, c->bf16, s);
    if (e == cudaSuccess) e = launch_plain_reduce(pa, false, s);
    if (grad && e == cudaSuccess) e = launch_plain_sample(pa, true, c->bf16, s);
    if (grad && e == cudaSuccess) e = launch_plain_reduce(pa, true, s);
    if (e != cudaSuccess) return cuda_fail(c, e, "plain-path launch");
  }
  if ((pe = prof_mark(c, 2, s)) != cudaSuccess) return cuda_fail(c, pe, "profile event");
  st = run_merge(c, K, 1, grad, d_lnL_event, d_neff_event, d_ln_xi, d_neff_sel, d_lnL_total,
                 d_flags, d_grad_total, s);
  if (st != GWC_OK) return st;
  if ((pe = prof_mark(c, 3, s)) != cudaSuccess) return cuda_fail(c, pe, "profile event");
  return GWC_OK;
}

gwc_status gwc_loglik_grad_host(gwc_ctx* c, int32_t K, const double* h_lambda,
                                double* h_lnL_total, int32_t* h_flags, double* h_grad_total,
                                void* stream) {
  if (!live(c)) return fail(nullptr, GWC_E_INVALID, "invalid or destroyed context");
  if (K < 1 || K > c->opt.max_K) return fail(c, GWC_E_INVALID, "K must be in [1, max_K]");
  if (!h_lambda || !h_lnL_total || !h_flags) return fail(c, GWC_E_INVALID, "NULL host pointer");
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  const size_t ne = (size_t)std::max(c->n_events, 1);
  double* lnL_event = c->d_out;
  double* neff_event = lnL_event + (size_t)c->opt.max_K * ne;
  double* ln_xi = neff_event + (size_t)c->opt.max_K * ne;
  double* neff_sel = ln_xi + c->opt.max_K;
  double* lnL_total = neff_sel + c->opt.max_K;
  double* grad = lnL_total + c->opt.max_K;
  std::memcpy(c->h_lam, h_lambda, sizeof(double) * (size_t)K * c->np);
  cudaError_t e = cudaMemcpyAsync(c->d_lam, c->h_lam, sizeof(double) * (size_t)K * c->np, cudaMemcpyHostToDevice, s);
  if (e != cudaSuccess) return cuda_fail(c, e, "H2D copy");
  gwc_status st = (h_grad_total ? gwc_loglik_grad(c, K, c->d_lam, lnL_event, neff_event, ln_xi, neff_sel,
                                                  lnL_total, c->d_flags, grad, stream)
                                : gwc_loglik(c, K, c->d_lam, lnL_event, neff_event, ln_xi, neff_sel,
                                             lnL_total, c->d_flags, stream));
  if (st != GWC_OK) return st;
  e = cudaMemcpyAsync(c->h_out, lnL_total, sizeof(double) * (size_t)K, cudaMemcpyDeviceToHost, s);
  if (e == cudaSuccess && h_grad_total)
    e = cudaMemcpyAsync(c->h_out + K, grad, sizeof(double) * (size_t)K * c->np, cudaMemcpyDeviceToHost, s);
  if (e == cudaSuccess)
    e = cudaMemcpyAsync(c->h_flags, c->d_flags, sizeof(int32_t) * (size_t)K, cudaMemcpyDeviceToHost, s);
  if (e == cudaSuccess) e = cudaStreamSynchronize(s);
  if (e != cudaSuccess) return cuda_fail(c, e, "D2H copy");
  std::memcpy(h_lnL_total, c->h_out, sizeof(double) * (size_t)K);
  std::memcpy(h_flags, c->h_flags, sizeof(int32_t) * (size_t)K);
  if (h_grad_total) std::memcpy(h_grad_total, c->h_out + K, sizeof(double) * (size_t)K * c->np);
  return GWC_OK;
}

void gwc_destroy(gwc_ctx* c) {
  if (!c) return;
  {
    std::lock_guard<std::mutex> g(g_mu);
    if (!g_live.count(c)) return;
    g_live.erase(c);
  }
  int cur = 0;
  cudaGetDevice(&cur);
  cudaSetDevice(c->device);
  free_all(c);
  cudaSetDevice(cur);
  c->magic = 0;
  delete c;
}

const char* gwc_last_error(const gwc_ctx* c) {
  if (c && live(c)) return c->err.c_str();
  return t_err.c_str();
}

gwc_status gwc_get_info(const gwc_ctx* c, gwc_info* out) {
  if (!live(c)) return fail(nullptr, GWC_E_INVALID, "invalid or destroyed context");
  if (!out) return GWC_E_INVALID;
  out->n_events = c->n_events;
  out->n_samples = c->n_samples;
  out->n_injections = c->n_inj;
  out->n_pix = c->n_pix;
  out->n_z = c->n_z;
  out->n_items = c->n_items;
  out->chunk = c->opt.chunk;
  out->n_x_table = c->opt.n_x_table;
  out->max_K = c->opt.max_K;
  out->device_bytes = c->device_bytes;
  out->n_params = c->np;
  out->mass_model = c->opt.mass_model;
  return GWC_OK;
}

gwc_status gwc_sample_terms(gwc_ctx* c, const double* d_lambda, float* d_lnw, float* d_dlnw,
                            double* d_c, int32_t* d_cell, void* stream) {
  if (!live(c)) return fail(nullptr, GWC_E_INVALID, "invalid or destroyed context");
  if (!d_lambda || !d_lnw || !d_c) return fail(c, GWC_E_INVALID, "NULL pointer");
  if (cudaSetDevice(c->device) != cudaSuccess) return fail(c, GWC_E_CUDA, "cudaSetDevice failed");
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  gwc_status st = run_prologue(c, 1, d_lambda, true, s);
  if (st != GWC_OK) return st;
  TermsArgs ta;
  ta.smp = c->smp;
  ta.pix = c->pix;
  ta.inj = c->inj;
  ta.los = c->los;
  ta.pbar32 = c->pbar32;
  ta.nz = c->n_z;
  ta.nx = c->opt.n_x_table;
  ta.n_samples = c->n_samples;
  ta.n_total = c->n_samples + c->n_inj;
  ta.lf = c->lf;
  ta.ld = c->ld;
  ta.tables = c->tables;
  ta.lnw = d_lnw;
  ta.dlnw = d_dlnw;
  ta.c = d_c;
  ta.mp = c->mp ? 1 : 0;
  ta.n_pix = c->n_pix;
  ta.cell = d_cell;
  cudaError_t e = launch_sample_terms(ta, c->bf16, s);
  if (e != cudaSuccess) return cuda_fail(c, e, "sample-terms launch");
  return GWC_OK;
}

gwc_status gwc_path_census(gwc_ctx* c, int32_t K, const double* d_lambda, uint64_t* d_counts, void* stream) {
  static_assert(GWC_CENSUS_N == GWC_CENSUS_SLOTS, "census slots");
  if (!live(c)) return fail(nullptr, GWC_E_INVALID, "invalid or destroyed context");
  if (K < 1 || K > c->opt.max_K) return fail(c, GWC_E_INVALID, "K must be in [1, max_K]");
  if (!d_lambda || !d_counts) return fail(c, GWC_E_INVALID, "NULL pointer");
  if (cudaSetDevice(c->device) != cudaSuccess) return fail(c, GWC_E_CUDA, "cudaSetDevice failed");
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  gwc_status st = run_prologue(c, K, d_lambda, false, s);
  if (st != GWC_OK) return st;
  CensusArgs ca;
  ca.smp = c->smp;
  ca.pix = c->pix;
  ca.inj = c->inj;
  ca.los = c->los;
  ca.pbar32 = c->pbar32;
  ca.nz = c->n_z;
  ca.nx = c->opt.n_x_table;
  ca.n_samples = c->n_samples;
  ca.n_total = c->n_samples + c->n_inj;
  ca.K = K;
  ca.lf = c->lf;
  ca.tables = c->tables;
  ca.tstride = c->tstride;
  ca.counts = reinterpret_cast<unsigned long long*>(d_counts);
  ca.mp = c->mp ? 1 : 0;
  cudaError_t e = launch_census(ca, c->bf16, s);
  if (e != cudaSuccess) return cuda_fail(c, e, "census launch");
  return GWC_OK;
}

gwc_status gwc_merge_parts(int32_t R, int32_t K, int32_t P, const double* parts, int32_t on_device,
                           double* lnL_total, double* ln_xi, double* neff_sel, int32_t* flags,
                           double* grad_total, void* stream) {
  if (R < 1 || K < 1) return fail(nullptr, GWC_E_INVALID, "R and K must be >= 1");
  if (P != 0 && P != NP && P != NP_MP) return fail(nullptr, GWC_E_INVALID, "P must be 0, 13 or 16");
  if (!parts || !lnL_total || !ln_xi || !neff_sel || !flags) return fail(nullptr, GWC_E_INVALID, "NULL pointer");
  if (!on_device) {
    for (int k = 0; k < K; ++k) merge_parts_point(R, K, P, parts, k, lnL_total, ln_xi, neff_sel, flags, grad_total);
    return GWC_OK;
  }
  const cudaError_t e = launch_merge_parts(R, K, P, parts, lnL_total, ln_xi, neff_sel, flags, grad_total,
                                           static_cast<cudaStream_t>(stream));
  if (e != cudaSuccess) return fail(nullptr, GWC_E_CUDA, std::string("merge_parts launch: ") + cudaGetErrorString(e));
  return GWC_OK;
}

gwc_status gwc_kde_census(gwc_ctx* c, int32_t K, const double* d_lambda, const gwc_kde_options* kopt,
                          uint64_t* d_counts, void* stream) {
  static_assert(GWC_KDE_CENSUS_N == KDE_CENSUS_SLOTS, "KDE census slots");
  if (!live(c)) return fail(nullptr, GWC_E_INVALID, "invalid or destroyed context");
  if (K < 1 || K > c->opt.max_K) return fail(c, GWC_E_INVALID, "K must be in [1, max_K]");
  if (!d_lambda || !d_counts) return fail(c, GWC_E_INVALID, "NULL pointer");
  gwc_kde_options ko;
  gwc_status st = kde_options_check(c, kopt, &ko);
  if (st != GWC_OK) return st;
  if (cudaSetDevice(c->device) != cudaSuccess) return fail(c, GWC_E_CUDA, "cudaSetDevice failed");
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  if ((st = kde_prepare(c, ko.n_grid, s)) != GWC_OK) return st;
  if ((st = run_prologue(c, K, d_lambda, false, s)) != GWC_OK) return st;
  cudaError_t e = cudaMemsetAsync(d_counts, 0, sizeof(uint64_t) * GWC_KDE_CENSUS_N, s);
  if (e != cudaSuccess) return cuda_fail(c, e, "census reset");
  KdeArgs ka = kde_args(c, ko, K);
  ka.census = reinterpret_cast<unsigned long long*>(d_counts);
  if ((e = launch_kde(ka, s)) != cudaSuccess) return cuda_fail(c, e, "KDE census launch");
  return GWC_OK;
}

struct gwc_graph {
  uint32_t magic = 0x67776367u;   // "gwcg"
  gwc_ctx* ctx = nullptr;
  uint64_t serial = 0;
  cudaGraphExec_t exec = nullptr;
};

namespace {
std::set<const gwc_graph*> g_graphs;
bool graph_live(const gwc_graph* g) {
  std::lock_guard<std::mutex> l(g_mu);
  return g && g_graphs.count(g) && g->magic == 0x67776367u;
}
}  // namespace

gwc_status gwc_graph_create(gwc_ctx* c, int32_t K, const double* d_lambda, int32_t want_grad,
                            double* d_lnL_event, double* d_neff_event, double* d_ln_xi,
                            double* d_neff_sel, double* d_lnL_total, int32_t* d_flags,
                            double* d_grad_total, gwc_graph** out) {
  if (!out) return fail(c, GWC_E_INVALID, "out is NULL");
  *out = nullptr;
  gwc_status st = check_call(c, K, d_lambda, d_lnL_event, d_neff_event, d_ln_xi, d_neff_sel,
                             d_lnL_total, d_flags);
  if (st != GWC_OK) return st;
  if (want_grad && !d_grad_total) return fail(c, GWC_E_INVALID, "d_grad_total is NULL");
  cudaStream_t cs = nullptr;
  cudaError_t e = cudaStreamCreateWithFlags(&cs, cudaStreamNonBlocking);
  if (e != cudaSuccess) return cuda_fail(c, e, "capture stream");
  // warm the occupancy cache outside the capture (it may set a kernel attribute)
  {
    int slab, n_slabs;
    fused_geometry(c, K, slab, n_slabs);
    FusedArgs fa{};
    fa.chunk = c->opt.chunk;
    fa.slab = slab;
    fa.group = group_for(c, K);
    fa.mp = c->mp ? 1 : 0;
    const bool grad = want_grad != 0, kahan = c->opt.accum == 1;
    const uint64_t key = ((uint64_t)fa.chunk << 20) | ((uint64_t)fa.slab << 8) | ((uint64_t)fa.group << 3) |
                         ((uint64_t)grad << 2) | ((uint64_t)kahan << 1) | (uint64_t)c->bf16;
    if (!c->occupancy.count(key)) {
      int bps = 0;
      e = fused_blocks_per_sm(fa, grad, kahan, c->bf16, &bps);
      if (e != cudaSuccess || bps < 1) {
        cudaStreamDestroy(cs);
        return e != cudaSuccess ? cuda_fail(c, e, "occupancy query")
                                : fail(c, GWC_E_UNSUPPORTED, "the fused kernel does not fit on an SM");
      }
      c->occupancy[key] = bps;
    }
  }
  e = cudaStreamBeginCapture(cs, cudaStreamCaptureModeThreadLocal);
  if (e != cudaSuccess) {
    cudaStreamDestroy(cs);
    return cuda_fail(c, e, "begin capture");
  }
  c->prof_off = true;
  st = run_fused(c, K, d_lambda, d_lnL_event, d_neff_event, d_ln_xi, d_neff_sel, d_lnL_total,
                 d_flags, want_grad ? d_grad_total : nullptr, want_grad != 0, cs);
  c->prof_off = false;
  cudaGraph_t graph = nullptr;
  e = cudaStreamEndCapture(cs, &graph);
  cudaStreamDestroy(cs);
  if (st != GWC_OK) {
    if (graph) cudaGraphDestroy(graph);
    return st;
  }
  if (e != cudaSuccess) return cuda_fail(c, e, "end capture");
  gwc_graph* g = new (std::nothrow) gwc_graph;
  if (!g) {
    cudaGraphDestroy(graph);
    return fail(c, GWC_E_NOMEM, "graph handle");
  }
  g->ctx = c;
  g->serial = c->serial;
  e = cudaGraphInstantiate(&g->exec, graph, 0);
  cudaGraphDestroy(graph);
  if (e != cudaSuccess) {
    delete g;
    return cuda_fail(c, e, "graph instantiate");
  }
  {
    std::lock_guard<std::mutex> l(g_mu);
    g_graphs.insert(g);
    ++c->live_recordings;
  }
  *out = g;
  return GWC_OK;
}

gwc_status gwc_graph_launch(gwc_graph* g, void* stream) {
  if (!graph_live(g)) return fail(nullptr, GWC_E_INVALID, "invalid or destroyed graph");
  gwc_ctx* c = g->ctx;
  if (!live(c) || c->serial != g->serial) return fail(nullptr, GWC_E_INVALID, "the graph's context was destroyed");
  if (cudaSetDevice(c->device) != cudaSuccess) return fail(c, GWC_E_CUDA, "cudaSetDevice failed");
  cudaError_t e = cudaGraphLaunch(g->exec, static_cast<cudaStream_t>(stream));
  if (e != cudaSuccess) return cuda_fail(c, e, "graph launch");
  return GWC_OK;
}

void gwc_graph_destroy(gwc_graph* g) {
  {
    std::lock_guard<std::mutex> l(g_mu);
    if (!g || !g_graphs.count(g)) return;
    g_graphs.erase(g);
    if (g_live.count(g->ctx) && g->ctx->serial == g->serial) --g->ctx->live_recordings;
  }
  if (g->exec) cudaGraphExecDestroy(g->exec);
  g->magic = 0;
  delete g;
}

struct gwc_hmc {
  uint32_t magic = 0x67776368u;   // "gwch"
  gwc_ctx* ctx = nullptr;
  uint64_t serial = 0;
  cudaGraphExec_t exec = nullptr;
  void* mem = nullptr;            // one device block: evaluation outputs and scratch
};

namespace {
std::set<const gwc_hmc*> g_hmcs;
bool hmc_live(const gwc_hmc* h) {
  std::lock_guard<std::mutex> l(g_mu);
  return h && g_hmcs.count(h) && h->magic == 0x67776368u;
}
}  // namespace

gwc_status gwc_hmc_create(gwc_ctx* c, int32_t K, int32_t n_leapfrog, const double* d_eps,
                          const double* d_inv_mass, double* d_q, double* d_p,
                          const double* d_log_u, double* d_lnL, double* d_grad,
                          int32_t* d_accept, double* d_H, gwc_hmc** out) {
  if (!out) return fail(c, GWC_E_INVALID, "out is NULL");
  *out = nullptr;
  if (!live(c)) return fail(nullptr, GWC_E_INVALID, "invalid or destroyed context");
  if (K < 1 || K > c->opt.max_K)
    return fail(c, GWC_E_INVALID, "K must be in [1, max_K] (max_K = " + std::to_string(c->opt.max_K) + ")");
  if (n_leapfrog < 1 || n_leapfrog > 4096) return fail(c, GWC_E_INVALID, "n_leapfrog must be in [1, 4096]");
  if (!d_eps || !d_inv_mass || !d_q || !d_p || !d_log_u || !d_lnL || !d_grad || !d_accept || !d_H)
    return fail(c, GWC_E_INVALID, "NULL device pointer");
  if (cudaSetDevice(c->device) != cudaSuccess) return fail(c, GWC_E_CUDA, "cudaSetDevice failed");
  gwc_hmc* h = new (std::nothrow) gwc_hmc;
  if (!h) return fail(c, GWC_E_NOMEM, "hmc handle");
  h->ctx = c;
  h->serial = c->serial;
  // device block: lnL_event, neff_event [K][n_ev]; ln_xi, neff_sel, lnL_total, lnL0 [K];
  // grad_total, q0, grad0 [K][np]; flags, div [K]
  const size_t ne = (size_t)std::max(c->n_events, 1);
  const size_t nd = 2 * (size_t)K * ne + 4 * (size_t)K + 3 * (size_t)K * c->np;
  cudaError_t e = cudaMalloc(&h->mem, nd * sizeof(double) + 2 * (size_t)K * sizeof(int32_t));
  if (e != cudaSuccess) {
    delete h;
    cudaGetLastError();
    return fail(c, e == cudaErrorMemoryAllocation ? GWC_E_NOMEM : GWC_E_CUDA,
                std::string("hmc scratch: ") + cudaGetErrorString(e));
  }
  double* m = static_cast<double*>(h->mem);
  double* lnL_event = m; m += (size_t)K * ne;
  double* neff_event = m; m += (size_t)K * ne;
  double* ln_xi = m; m += K;
  double* neff_sel = m; m += K;
  double* lnL_total = m; m += K;
  double* lnL0 = m; m += K;
  double* grad_total = m; m += (size_t)K * c->np;
  double* q0 = m; m += (size_t)K * c->np;
  double* grad0 = m; m += (size_t)K * c->np;
  int32_t* flags = reinterpret_cast<int32_t*>(m);
  int32_t* div = flags + K;

  HmcArgs ha;
  ha.K = K;
  ha.np = c->np;
  ha.eps = d_eps;
  ha.inv_mass = d_inv_mass;
  ha.q = d_q;
  ha.p = d_p;
  ha.q0 = q0;
  ha.lnL0 = lnL0;
  ha.grad0 = grad0;
  ha.div = div;
  ha.lnL = lnL_total;
  ha.grad = grad_total;
  ha.flags = flags;
  ha.log_u = d_log_u;
  ha.H = d_H;
  ha.accept = d_accept;
  ha.lnL_out = d_lnL;
  ha.grad_out = d_grad;

  cudaStream_t cs = nullptr;
  e = cudaStreamCreateWithFlags(&cs, cudaStreamNonBlocking);
  if (e != cudaSuccess) {
    cudaFree(h->mem);
    delete h;
    return cuda_fail(c, e, "capture stream");
  }
  // occupancy of the gradient kernel, outside the capture
  gwc_status st = GWC_OK;
  {
    int slab, n_slabs;
    fused_geometry(c, K, slab, n_slabs);
    FusedArgs fa{};
    fa.chunk = c->opt.chunk;
    fa.slab = slab;
    fa.group = group_for(c, K);
    fa.mp = c->mp ? 1 : 0;
    const bool kahan = c->opt.accum == 1;
    const uint64_t key = ((uint64_t)fa.chunk << 20) | ((uint64_t)fa.slab << 8) | ((uint64_t)fa.group << 3) |
                         (1ull << 2) | ((uint64_t)kahan << 1) | (uint64_t)c->bf16;
    if (!c->occupancy.count(key)) {
      int bps = 0;
      e = fused_blocks_per_sm(fa, true, kahan, c->bf16, &bps);
      if (e != cudaSuccess) st = cuda_fail(c, e, "occupancy query");
      else if (bps < 1) st = fail(c, GWC_E_UNSUPPORTED, "the fused kernel does not fit on an SM");
      else c->occupancy[key] = bps;
    }
  }
  cudaGraph_t graph = nullptr;
  if (st == GWC_OK) {
    e = cudaStreamBeginCapture(cs, cudaStreamCaptureModeThreadLocal);
    if (e != cudaSuccess) st = cuda_fail(c, e, "begin capture");
  }
  if (st == GWC_OK) {
    c->prof_off = true;
    auto eval = [&]() {
      return run_fused(c, K, d_q, lnL_event, neff_event, ln_xi, neff_sel, lnL_total, flags,
                       grad_total, true, cs);
    };
    auto stage = [&](int mode) {
      ha.mode = mode;
      cudaError_t r = launch_hmc(ha, cs);
      return r == cudaSuccess ? GWC_OK : cuda_fail(c, r, "leapfrog launch");
    };
    st = stage(0);
    if (st == GWC_OK) st = eval();
    if (st == GWC_OK) st = stage(1);
    for (int l = 1; l < n_leapfrog && st == GWC_OK; ++l) {
      st = eval();
      if (st == GWC_OK) st = stage(2);
    }
    if (st == GWC_OK) st = eval();
    if (st == GWC_OK) st = stage(3);
    c->prof_off = false;
    e = cudaStreamEndCapture(cs, &graph);
    if (st == GWC_OK && e != cudaSuccess) st = cuda_fail(c, e, "end capture");
  }
  cudaStreamDestroy(cs);
  if (st == GWC_OK) {
    e = cudaGraphInstantiate(&h->exec, graph, 0);
    if (e != cudaSuccess) st = cuda_fail(c, e, "graph instantiate");
  }
  if (graph) cudaGraphDestroy(graph);
  if (st != GWC_OK) {
    cudaFree(h->mem);
    delete h;
    return st;
  }
  {
    std::lock_guard<std::mutex> l(g_mu);
    g_hmcs.insert(h);
    ++c->live_recordings;
  }
  *out = h;
  return GWC_OK;
}

gwc_status gwc_hmc_launch(gwc_hmc* h, void* stream) {
  if (!hmc_live(h)) return fail(nullptr, GWC_E_INVALID, "invalid or destroyed hmc object");
  gwc_ctx* c = h->ctx;
  if (!live(c) || c->serial != h->serial) return fail(nullptr, GWC_E_INVALID, "the hmc object's context was destroyed");
  if (cudaSetDevice(c->device) != cudaSuccess) return fail(c, GWC_E_CUDA, "cudaSetDevice failed");
  cudaError_t e = cudaGraphLaunch(h->exec, static_cast<cudaStream_t>(stream));
  if (e != cudaSuccess) return cuda_fail(c, e, "trajectory launch");
  return GWC_OK;
}

void gwc_hmc_destroy(gwc_hmc* h) {
  {
    std::lock_guard<std::mutex> l(g_mu);
    if (!h || !g_hmcs.count(h)) return;
    g_hmcs.erase(h);
    if (g_live.count(h->ctx) && h->ctx->serial == h->serial) --h->ctx->live_recordings;
  }
  if (h->exec) cudaGraphExecDestroy(h->exec);
  if (h->mem) cudaFree(h->mem);
  h->magic = 0;
  delete h;
}

gwc_status gwc_autotune(gwc_ctx* c, int32_t K, const double* d_lambda, int32_t want_grad,
                        void* stream, gwc_tune_result* out) {
  if (!live(c)) return fail(nullptr, GWC_E_INVALID, "invalid or destroyed context");
  if (K < 1 || K > c->opt.max_K)
    return fail(c, GWC_E_INVALID, "K must be in [1, max_K] (max_K = " + std::to_string(c->opt.max_K) + ")");
  if (!d_lambda) return fail(c, GWC_E_INVALID, "d_lambda is NULL");
  {
    std::lock_guard<std::mutex> l(g_mu);
    if (c->live_recordings > 0)
      return fail(c, GWC_E_INVALID, "destroy the context's graphs and HMC objects before tuning");
  }
  if (cudaSetDevice(c->device) != cudaSuccess) return fail(c, GWC_E_CUDA, "cudaSetDevice failed");
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  cudaError_t e = cudaDeviceSynchronize();
  if (e != cudaSuccess) return cuda_fail(c, e, "synchronise before tuning");
  const size_t ne = (size_t)std::max(c->n_events, 1);
  double* tmp = nullptr;
  int32_t* fl = nullptr;
  cudaEvent_t e0 = nullptr, e1 = nullptr;
  e = cudaMalloc(reinterpret_cast<void**>(&tmp), sizeof(double) * (2 * (size_t)K * ne + 3 * (size_t)K + (size_t)K * c->np));
  if (e == cudaSuccess) e = cudaMalloc(reinterpret_cast<void**>(&fl), sizeof(int32_t) * (size_t)K);
  if (e == cudaSuccess) e = cudaEventCreate(&e0);
  if (e == cudaSuccess) e = cudaEventCreate(&e1);
  auto release = [&]() {
    if (tmp) cudaFree(tmp);
    if (fl) cudaFree(fl);
    if (e0) cudaEventDestroy(e0);
    if (e1) cudaEventDestroy(e1);
  };
  if (e != cudaSuccess) {
    release();
    cudaGetLastError();
    return cuda_fail(c, e, "tuning scratch");
  }
  double* lnL_event = tmp;
  double* neff_event = lnL_event + (size_t)K * ne;
  double* ln_xi = neff_event + (size_t)K * ne;
  double* neff_sel = ln_xi + K;
  double* lnL_total = neff_sel + K;
  double* grad = lnL_total + K;
  const bool g = want_grad != 0;
  const gwc_options keep = c->opt;
  gwc_tune_result best{keep.chunk, keep.lambda_tile, keep.lambda_group, 0, INFINITY};
  int n_tried = 0;
  gwc_status st = GWC_OK;
  c->prof_off = true;
  const int chunks[] = {1024, 1536, 2048};
  const int tiles[] = {16, 32, 64, 128, 256};
  const int groups[] = {1, 2, 4, 8};
  for (int chunk : chunks) {
    if (st != GWC_OK) break;
    st = set_chunk(c, chunk);
    int last_tile = -1;
    for (int tile : tiles) {
      const int t = std::min(tile, (int)K);
      if (st != GWC_OK || t == last_tile) continue;
      last_tile = t;
      for (int grp : groups) {
        if (t * grp > MAX_SLAB_GROUP) continue;   // the geometry would cut the tile
        c->opt.lambda_tile = t;
        c->opt.lambda_group = grp;
        auto run = [&]() {
          return run_fused(c, K, d_lambda, lnL_event, neff_event, ln_xi, neff_sel, lnL_total, fl,
                           g ? grad : nullptr, g, s);
        };
        st = run();
        if (st == GWC_OK && (e = cudaEventRecord(e0, s)) != cudaSuccess) st = cuda_fail(c, e, "event");
        if (st == GWC_OK) st = run();
        if (st == GWC_OK) st = run();
        if (st == GWC_OK && (e = cudaEventRecord(e1, s)) != cudaSuccess) st = cuda_fail(c, e, "event");
        float ms = 0.f;
        if (st == GWC_OK && (e = cudaEventSynchronize(e1)) != cudaSuccess) st = cuda_fail(c, e, "tuning run");
        if (st == GWC_OK && (e = cudaEventElapsedTime(&ms, e0, e1)) != cudaSuccess) st = cuda_fail(c, e, "event");
        if (st != GWC_OK) break;
        ++n_tried;
        if (0.5 * ms < best.ms) best = gwc_tune_result{chunk, t, grp, 0, 0.5 * (double)ms};
      }
    }
  }
  c->prof_off = false;
  release();
  if (st != GWC_OK) {
    cudaDeviceSynchronize();
    cudaGetLastError();
    set_chunk(c, keep.chunk);
    c->opt.lambda_tile = keep.lambda_tile;
    c->opt.lambda_group = keep.lambda_group;
    return st;
  }
  st = set_chunk(c, best.chunk);
  if (st != GWC_OK) return st;
  c->opt.lambda_tile = best.lambda_tile;
  c->opt.lambda_group = best.lambda_group;
  best.n_tried = n_tried;
  if (out) *out = best;
  return GWC_OK;
}

gwc_status gwc_profile_enable(gwc_ctx* c, int32_t enable) {
  if (!live(c)) return fail(nullptr, GWC_E_INVALID, "invalid or destroyed context");
  if (cudaSetDevice(c->device) != cudaSuccess) return fail(c, GWC_E_CUDA, "cudaSetDevice failed");
  if (enable && c->prof_ev.empty()) {
    c->prof_ev.assign((size_t)PROF_SLOTS * 4, nullptr);
    for (auto& e : c->prof_ev) {
      cudaError_t r = cudaEventCreate(&e);
      if (r != cudaSuccess) {
        for (auto& x : c->prof_ev)
          if (x) cudaEventDestroy(x);
        c->prof_ev.clear();
        return cuda_fail(c, r, "cudaEventCreate");
      }
    }
    c->prof_used = 0;
    c->prof_calls = 0;
    for (double& m : c->prof_ms) m = 0.0;
  } else if (!enable && !c->prof_ev.empty()) {
    cudaError_t r = prof_drain(c);
    for (auto& e : c->prof_ev) cudaEventDestroy(e);
    c->prof_ev.clear();
    if (r != cudaSuccess) return cuda_fail(c, r, "profile drain");
  }
  return GWC_OK;
}

gwc_status gwc_profile_read(gwc_ctx* c, double* ms, int64_t* n_calls) {
  if (!live(c)) return fail(nullptr, GWC_E_INVALID, "invalid or destroyed context");
  if (!ms || !n_calls) return fail(c, GWC_E_INVALID, "NULL output");
  if (!c->prof_ev.empty()) {
    cudaError_t r = prof_drain(c);
    if (r != cudaSuccess) return cuda_fail(c, r, "profile drain");
  }
  for (int i = 0; i < 3; ++i) {
    ms[i] = c->prof_ms[i];
    c->prof_ms[i] = 0.0;
  }
  *n_calls = c->prof_calls;
  c->prof_calls = 0;
  return GWC_OK;
}

gwc_status gwc_los_cell_index(const float* d_z, int64_t n, int32_t n_z, double z_max,
                              int32_t* d_cell, void* stream) {
  if (n < 0 || n_z < 2 || !(z_max > 0.0) || (n > 0 && (!d_z || !d_cell)))
    return fail(nullptr, GWC_E_INVALID, "bad arguments");
  cudaError_t e = launch_los_cell(d_z, n, n_z, z_max, d_cell, static_cast<cudaStream_t>(stream));
  if (e != cudaSuccess) return cuda_fail(nullptr, e, "cell-index launch");
  return GWC_OK;
}

}  // extern "C"
