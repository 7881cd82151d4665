// gwc_api.cu -- the C ABI (include/gwc.h): validation, device layout, launch sequences.
//
// Device layout built by gwc_create:
//   samples      float4 {m1_det, m2_det, d_L, ln pi_PE} + int32 pixel, sorted by event
//                and, within an event, by pixel (so a chunk touches few LOS rows)
//   injections   float4 {m1_det, m2_det, d_L, ln p_draw}
//   LOS table    [n_pix][n_z] float (or bfloat16); the pixel mean in float and double
//   work items   runs of <= chunk samples of one event (events split evenly), then runs
//                of injections; launched largest first
// Per call (sized for max_K at create, so calls allocate nothing):
//   per-Lambda constants and tables, and the partial sums [K][items][parts][16].
#include <algorithm>
#include <cmath>
#include <cstdio>
#include <cstring>
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
  double* ev_n = nullptr;
  LamF* lf = nullptr;
  LamD* ld = nullptr;
  float* tables = nullptr;
  float* partials = nullptr;
  // host-call staging
  double* d_lam = nullptr;
  double* d_out = nullptr;      // lnL_event, neff_event, ln_xi, neff_sel, lnL_total, grad
  int32_t* d_flags = nullptr;
  double* h_lam = nullptr;      // pinned
  double* h_out = nullptr;      // pinned: lnL_total[K], grad[K][13]
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
                 c->ev_item0, c->ev_n, c->lf, c->ld, c->tables, c->partials, c->d_lam, c->d_out,
                 c->d_flags, c->sample_item, c->plain_lw, c->plain_tg};
  for (void* p : dev)
    if (p) cudaFree(p);
  if (c->h_lam) cudaFreeHost(c->h_lam);
  if (c->h_out) cudaFreeHost(c->h_out);
  if (c->h_flags) cudaFreeHost(c->h_flags);
}

constexpr int PROF_SLOTS = 256;

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
  if (c->prof_ev.empty()) return cudaSuccess;
  if (b == 0 && c->prof_used == PROF_SLOTS) {
    cudaError_t r = prof_drain(c);
    if (r != cudaSuccess) return r;
  }
  cudaError_t r = cudaEventRecord(prof_event(c, b), s);
  if (b == 3 && r == cudaSuccess) ++c->prof_used;
  return r;
}

void gauss_legendre(int n, double* x, double* w) {
  const double pi = 3.14159265358979323846;
  for (int i = 0; i < n; ++i) {
    double z = std::cos(pi * (i + 0.75) / (n + 0.5)), dp = 1.0;
    for (int it = 0; it < 100; ++it) {
      double p0 = 1.0, p1 = z;
      for (int j = 2; j <= n; ++j) {
        const double p2 = ((2.0 * j - 1.0) * z * p1 - (j - 1.0) * p0) / j;
        p0 = p1;
        p1 = p2;
      }
      dp = n * (z * p1 - p0) / (z * z - 1.0);
      const double dz = p1 / dp;
      z -= dz;
      if (std::fabs(dz) < 1e-16) break;
    }
    x[i] = z;
    w[i] = 2.0 / ((1.0 - z * z) * dp * dp);
  }
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

// launch geometry of the fused kernel for a batch of K points
void fused_geometry(const gwc_ctx* c, int K, int& slab, int& n_slabs) {
  slab = c->opt.lambda_tile > 0 ? c->opt.lambda_tile : 64;
  slab = std::max(1, std::min(std::min(slab, K), MAX_SLAB));
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

gwc_status run_prologue(gwc_ctx* c, int K, const double* d_lambda, bool grad, cudaStream_t s) {
  ProArgs pa;
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
  cudaError_t e = launch_prologue(pa, K, s);
  if (e != cudaSuccess) return cuda_fail(c, e, "prologue launch");
  return GWC_OK;
}

gwc_status run_merge(gwc_ctx* c, int K, int P, bool grad, double* lnL_event, double* neff_event,
                     double* ln_xi, double* neff_sel, double* lnL_total, int32_t* flags,
                     double* grad_total, cudaStream_t s) {
  MergeArgs ma;
  ma.partials = c->partials;
  ma.n_items = c->n_items;
  ma.P = P;
  ma.ev_item0 = c->ev_item0;
  ma.n_events = c->n_events;
  ma.inj_item0 = c->inj_item0;
  ma.ev_n = c->ev_n;
  ma.n_draw = c->n_draw;
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

gwc_status run_fused(gwc_ctx* c, int32_t K, const double* d_lambda, double* lnL_event,
                     double* neff_event, double* ln_xi, double* neff_sel, double* lnL_total,
                     int32_t* flags, double* grad_total, bool grad, cudaStream_t s) {
  cudaError_t pe = prof_mark(c, 0, s);
  if (pe != cudaSuccess) return cuda_fail(c, pe, "profile event");
  gwc_status st = run_prologue(c, K, d_lambda, grad, s);
  if (st != GWC_OK) return st;
  if ((pe = prof_mark(c, 1, s)) != cudaSuccess) return cuda_fail(c, pe, "profile event");
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
  fa.sched = c->sched;
  fa.n_items = c->n_items;
  fa.n_slabs = n_slabs;
  fa.slab = slab;
  fa.group = c->opt.lambda_group > 0 ? c->opt.lambda_group : 2;
  fa.K = K;
  fa.chunk = c->opt.chunk;
  fa.lf = c->lf;
  fa.tables = c->tables;
  fa.tstride = c->tstride;
  fa.partials = c->partials;
  const long long grid = (long long)c->n_items * n_slabs;
  if (grid > 0x7fffffffLL) return fail(c, GWC_E_INVALID, "work grid too large");
  cudaError_t e = launch_fused(fa, grad, c->opt.accum == 1, c->bf16, (int)grid, s);
  if (e != cudaSuccess) return cuda_fail(c, e, "sample kernel launch");
  if ((e = prof_mark(c, 2, s)) != cudaSuccess) return cuda_fail(c, e, "profile event");
  st = run_merge(c, K, 1, grad, lnL_event, neff_event, ln_xi, neff_sel, lnL_total, flags,
                 grad_total, s);
  if (st != GWC_OK) return st;
  if ((e = prof_mark(c, 3, s)) != cudaSuccess) return cuda_fail(c, e, "profile event");
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

  // ---- validate the events
  const int32_t ne = ev->n_events;
  if (ne < 0) return fail(nullptr, GWC_E_INVALID, "n_events < 0");
  if (!ev->offsets) return fail(nullptr, GWC_E_INVALID, "offsets is NULL");
  if (ev->offsets[0] != 0) return fail(nullptr, GWC_E_INVALID, "offsets[0] must be 0");
  for (int32_t e = 0; e < ne; ++e)
    if (ev->offsets[e + 1] <= ev->offsets[e])
      return fail(nullptr, GWC_E_INVALID, "offsets must be strictly increasing (event " + std::to_string(e) + ")");
  const int64_t ns = ev->offsets[ne];
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
  std::vector<Item> items;
  std::vector<int32_t> ev_item0((size_t)ne + 1);
  std::vector<double> ev_n((size_t)std::max(ne, 1));
  for (int32_t e = 0; e < ne; ++e) {
    ev_item0[(size_t)e] = (int32_t)items.size();
    split_items(ev->offsets[e], ev->offsets[e + 1] - ev->offsets[e], o.chunk, 0, items);
    ev_n[(size_t)e] = (double)(ev->offsets[e + 1] - ev->offsets[e]);
  }
  ev_item0[(size_t)ne] = (int32_t)items.size();
  c->inj_item0 = (int32_t)items.size();
  split_items(0, ni, o.chunk, 1, items);
  if (items.size() > 0x7fffffffu) { delete c; return fail(nullptr, GWC_E_INVALID, "too many work items"); }
  c->n_items = (int32_t)items.size();
  std::vector<int32_t> sched((size_t)c->n_items);
  for (int32_t i = 0; i < c->n_items; ++i) sched[(size_t)i] = i;
  std::stable_sort(sched.begin(), sched.end(),
                   [&](int32_t a, int32_t b) { return items[(size_t)a].count > items[(size_t)b].count; });
  c->h_sample_item.assign((size_t)(ns + ni), 0);
  for (int32_t i = 0; i < c->n_items; ++i) {
    const Item& it = items[(size_t)i];
    const int64_t base = it.kind == 1 ? ns + it.begin : it.begin;
    for (int32_t q = 0; q < it.count; ++q) c->h_sample_item[(size_t)(base + q)] = i;
  }
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
  chk(dalloc(c, &c->ev_n, ev_n.size()));
  chk(dalloc(c, &c->lf, (size_t)o.max_K));
  chk(dalloc(c, &c->ld, (size_t)o.max_K));
  chk(dalloc(c, &c->tables, (size_t)o.max_K * c->tstride));
  chk(dalloc(c, &c->partials, (size_t)kcap * c->n_items * PSTRIDE));
  chk(dalloc(c, &c->d_lam, (size_t)o.max_K * NP));
  chk(dalloc(c, &c->d_out, (size_t)o.max_K * (2 * (size_t)std::max(ne, 1) + 3 + NP)));
  chk(dalloc(c, &c->d_flags, (size_t)o.max_K));
  if (e == cudaSuccess) e = cudaMallocHost(reinterpret_cast<void**>(&c->h_lam), sizeof(double) * o.max_K * NP);
  if (e == cudaSuccess) e = cudaMallocHost(reinterpret_cast<void**>(&c->h_out), sizeof(double) * o.max_K * (1 + NP));
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
  chk(cudaMemcpy(c->ev_n, ev_n.data(), sizeof(double) * ev_n.size(), cudaMemcpyHostToDevice));
  double glx[NGL], glw[NGL];
  gauss_legendre(NGL, glx, glw);
  chk(set_gauss_legendre(glx, glw));
  if (e != cudaSuccess) {
    std::string msg = std::string("device upload failed: ") + cudaGetErrorString(e);
    free_all(c);
    delete c;
    return fail(nullptr, GWC_E_CUDA, msg);
  }
  {
    std::lock_guard<std::mutex> g(g_mu);
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

gwc_status gwc_loglik_plain(gwc_ctx* c, int32_t K, const double* d_lambda, double* d_lnL_event,
                            double* d_neff_event, double* d_ln_xi, double* d_neff_sel,
                            double* d_lnL_total, int32_t* d_flags, double* d_grad_total,
                            void* stream) {
  gwc_status st = check_call(c, K, d_lambda, d_lnL_event, d_neff_event, d_ln_xi, d_neff_sel,
                             d_lnL_total, d_flags);
  if (st != GWC_OK) return st;
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
  std::memcpy(c->h_lam, h_lambda, sizeof(double) * (size_t)K * NP);
  cudaError_t e = cudaMemcpyAsync(c->d_lam, c->h_lam, sizeof(double) * (size_t)K * NP, cudaMemcpyHostToDevice, s);
  if (e != cudaSuccess) return cuda_fail(c, e, "H2D copy");
  gwc_status st = (h_grad_total ? gwc_loglik_grad(c, K, c->d_lam, lnL_event, neff_event, ln_xi, neff_sel,
                                                  lnL_total, c->d_flags, grad, stream)
                                : gwc_loglik(c, K, c->d_lam, lnL_event, neff_event, ln_xi, neff_sel,
                                             lnL_total, c->d_flags, stream));
  if (st != GWC_OK) return st;
  e = cudaMemcpyAsync(c->h_out, lnL_total, sizeof(double) * (size_t)K, cudaMemcpyDeviceToHost, s);
  if (e == cudaSuccess && h_grad_total)
    e = cudaMemcpyAsync(c->h_out + K, grad, sizeof(double) * (size_t)K * NP, cudaMemcpyDeviceToHost, s);
  if (e == cudaSuccess)
    e = cudaMemcpyAsync(c->h_flags, c->d_flags, sizeof(int32_t) * (size_t)K, cudaMemcpyDeviceToHost, s);
  if (e == cudaSuccess) e = cudaStreamSynchronize(s);
  if (e != cudaSuccess) return cuda_fail(c, e, "D2H copy");
  std::memcpy(h_lnL_total, c->h_out, sizeof(double) * (size_t)K);
  std::memcpy(h_flags, c->h_flags, sizeof(int32_t) * (size_t)K);
  if (h_grad_total) std::memcpy(h_grad_total, c->h_out + K, sizeof(double) * (size_t)K * NP);
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
  return GWC_OK;
}

gwc_status gwc_sample_terms(gwc_ctx* c, const double* d_lambda, float* d_lnw, float* d_dlnw,
                            double* d_c, void* stream) {
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
  cudaError_t e = launch_sample_terms(ta, c->bf16, s);
  if (e != cudaSuccess) return cuda_fail(c, e, "sample-terms launch");
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
