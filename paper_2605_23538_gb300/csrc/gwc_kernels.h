// gwc_kernels.h -- launch interface between the host API (gwc_api.cu) and the kernels.
#pragma once

#include <cstddef>
#include <cstdint>
#include <string>
#include <cuda_runtime.h>

#include "gwc_internal.cuh"

namespace gwc {

struct ProArgs {
  const double* lam;      // [K][13], or [K][16] for the multi-peak model
  int mp = 0;             // mass model: 0 power law + peak, 1 multi-peak
  int nx;                 // nodes of the inversion table
  int nz;                 // LOS grid nodes
  double zmax;
  const double* pbar64;   // [nz] pixel-averaged LOS prior (FP64)
  LamF* lf;               // [K]
  LamD* ld;               // [K]
  float* tables;          // [K][tstride]
  int tstride;
  int want_grad;
  int* counter = nullptr;   // zeroed by CTA 0 when set (the fused kernel's work counter)
  int32_t* order = nullptr; // when set: order[r] = the Lambda point of rank r by H0 (the
                            // order in which the fused kernel takes points)
};

struct FusedArgs {
  const float4* smp;      // event samples {m1, m2, dL, ln pi}
  const int32_t* pix;
  const float4* inj;      // injections {m1, m2, dL, ln p_draw}
  const void* los;        // [n_pix][nz] float or bf16
  const float* pbar32;    // [nz]
  int nz;
  int nx;
  const Item* items;      // canonical order: events' items, then injection items
  const int32_t* sched;   // launch order (largest items first)
  int n_items;
  int n_slabs;            // Lambda tiles per item
  int slab;               // Lambda points per tile (<= MAX_SLAB)
  int group;              // warps sharing one Lambda point: 1, 2, 4 or 8
  int K;
  int chunk;
  const LamF* lf;
  const float* tables;
  int tstride;
  float* partials;        // [K][stride][PSTRIDE], slot slot0 + item
  int* counter;           // next (item, slab) unit; zero at launch
  const int32_t* order;   // Lambda points in the order taken (by H0), or null (index order)
  int n_sched;            // schedule entries (units = n_sched * n_slabs)
  int stride;             // partial slots per Lambda
  int slot0;              // slot of item 0
  int mp = 0;             // multi-peak mass model
};

// KDE form of the event term: one (event, pixel) group of samples
struct KdeGroup {
  int64_t begin;
  int32_t count;
  int32_t pix;
};

struct KdeArgs {
  const float4* smp;
  const float2* lm;       // log2 m1_det, log2 m2_det of every sample
  const KdeGroup* groups;
  int n_groups;
  const float* pgrid;     // [n_pix][kde_row(G)]: the LOS prior at the KDE grid points, rows
                          // padded with zeros to whole blocks of KDE_BLOCK floats
  int G;
  float dzg;              // grid step z_max / (G - 1)
  int rule;               // 0 Scott, 1 Silverman, 2 biweight
  float neff_min;         // per-pixel N_eff threshold
  int K;
  int nx, nz;
  const LamF* lf;
  const float* tables;
  int tstride;
  float* partials;        // [K][stride][PSTRIDE], slot = group index
  int stride;
  int mp = 0;             // multi-peak mass model
  // measurement only (null otherwise): [0] pass-1 sample evaluations, [1] (group, Lambda)
  // pairs kept, [2] pass-2 sample evaluations with a weight, [3] grid terms summed
  unsigned long long* census = nullptr;
};
constexpr int KDE_CENSUS_SLOTS = 4;
// a KDE grid row's stride: the grid points rounded up to whole blocks of 4 (16 bytes)
constexpr int KDE_BLOCK = 4;
__host__ __device__ constexpr int kde_row(int G) { return (G + KDE_BLOCK - 1) / KDE_BLOCK * KDE_BLOCK; }
cudaError_t launch_kde(const KdeArgs& a, cudaStream_t s);
cudaError_t launch_log2_masses(const float4* smp, long long n, float2* out, cudaStream_t s);
cudaError_t launch_los_grid(const float* los, int n_pix, int nz, double zmax, int G, float* out,
                            cudaStream_t s);

struct PlainArgs {
  const float4* smp;
  const int32_t* pix;
  const float4* inj;
  const void* los;
  const float* pbar32;
  int nz;
  int nx;
  long long n_samples;
  long long n_total;      // samples + injections
  const Item* items;
  const int32_t* sample_item;   // [n_total] item of each sample / injection
  int n_items;
  int k;                  // the Lambda point of this pass
  const LamF* lf;
  const float* tables;
  int tstride;
  float* lw;              // [n_total]
  float* tg;              // [13][n_total]
  float* partials;        // [K][n_items][1][PSTRIDE]
};

struct MergeArgs {
  int mp = 0;               // multi-peak mass model: 16 gradient components, else 13
  const float* partials;
  int n_items;
  int P;
  const int32_t* ev_item0;  // [n_events + 1]
  int n_events;
  int inj_item0;
  const double* ln_ev_n;    // [n_events] ln of the samples per event, N_i
  double ln_n_draw;         // ln of the injection draws
  const LamD* ld;
  double neff_min_event;
  double neff_min_sel;
  double* lnL_event;
  double* neff_event;
  double* ln_xi;
  double* neff_sel;
  double* lnL_total;
  int32_t* flags;
  double* grad_total;
  // optional parts for merging shards of a catalogue (may be null): sum_i ln L_i [K],
  // its gradient [K][P], and the gradient of ln xi [K][P] (P = 13, or 16 multi-peak)
  double* sum_events = nullptr;
  double* grad_events = nullptr;
  double* grad_ln_xi = nullptr;
};

// One leapfrog stage of K Hamiltonian Monte Carlo chains (one warp per chain, a lane
// per parameter).  mode 0: save q0, clear the divergence mark.  1: after the evaluation
// at q0: record lnL0, grad0 and H0 = -lnL + p.M^-1.p / 2, then half kick and drift.
// 2: full kick and drift.  3: final half kick, H1, and the Metropolis decision.
struct HmcArgs {
  int K;
  int mode;
  int np;                   // parameters per chain (13, or 16 multi-peak): P below
  const double* eps;        // [K] step sizes
  const double* inv_mass;   // [P] diagonal inverse mass
  double* q;                // [K][P] position (in/out)
  double* p;                // [K][P] momentum (in/out)
  double* q0;               // [K][P] scratch
  double* lnL0;             // [K] scratch
  double* grad0;            // [K][P] scratch
  int32_t* div;             // [K] scratch: the chain met a flagged (invalid) point
  const double* lnL;        // [K] the last evaluation
  const double* grad;       // [K][P]
  const int32_t* flags;     // [K]
  const double* log_u;      // [K] log of a uniform(0, 1) number per chain
  double* H;                // [K][2] Hamiltonian at the start and the end
  int32_t* accept;          // [K]
  double* lnL_out;          // [K] log-likelihood at the returned position
  double* grad_out;         // [K][P]
};
cudaError_t launch_hmc(const HmcArgs& a, cudaStream_t s);

// the prologue's per-device setup, once per device and outside any stream capture: its
// Gauss-Legendre constants, and permission for its 16-CTA cluster shape
cudaError_t ensure_prologue_ready();
cudaError_t launch_prologue(const ProArgs& a, int K, cudaStream_t s);
constexpr int MAX_SLAB = 256;        // Lambda points per CTA tile at most
constexpr int MAX_SLAB_GROUP = 512;  // tile points x warps per point at most (the combine's
                                     // shared memory: this many partials of PSTRIDE floats)
size_t fused_smem_bytes(int chunk, int slab, int group, bool grad);
size_t fused_smem_max();
cudaError_t launch_fused(const FusedArgs& a, bool grad, bool kahan, bool bf16, int grid, cudaStream_t s);
// CTAs of the fused kernel that fit on one SM at this geometry (occupancy query)
cudaError_t fused_blocks_per_sm(const FusedArgs& a, bool grad, bool kahan, bool bf16, int* out);
cudaError_t launch_plain_sample(const PlainArgs& a, bool grad, bool bf16, cudaStream_t s);
cudaError_t launch_plain_reduce(const PlainArgs& a, bool grad, cudaStream_t s);
cudaError_t launch_merge(const MergeArgs& a, int K, bool grad, cudaStream_t s);
struct TermsArgs {
  const float4* smp;
  const int32_t* pix;
  const float4* inj;
  const void* los;
  const float* pbar32;
  int nz;
  int nx;
  long long n_samples;
  long long n_total;
  const LamF* lf;
  const LamD* ld;
  const float* tables;
  float* lnw;       // [n_total]
  float* dlnw;      // [P][n_total] or nullptr (P = 13, or 16 multi-peak)
  double* c;        // [1 + P]
  int mp = 0;       // multi-peak mass model
  int n_pix = 0;    // rows of los: a sample whose pixel lies outside [0, n_pix) gets w = 0
  int32_t* cell = nullptr;   // [n_total] or nullptr: the LOS cell each sample interpolates in
};
cudaError_t launch_sample_terms(const TermsArgs& a, bool bf16, cudaStream_t s);
constexpr int GWC_CENSUS_SLOTS = 10;
struct CensusArgs {
  const float4* smp;
  const int32_t* pix;
  const float4* inj;
  const void* los;
  const float* pbar32;
  int nz;
  int nx;
  long long n_samples;
  long long n_total;
  int K;
  const LamF* lf;
  const float* tables;
  int tstride;
  unsigned long long* counts;   // [GWC_CENSUS_SLOTS], zeroed by the launcher
  int mp = 0;
};
cudaError_t launch_census(const CensusArgs& a, bool bf16, cudaStream_t s);
// Combination of event shards' parts for one Lambda point k (host or device, FP64, ranks
// in order).  parts[R][K][5 + 2P]: sum of the shard's ln L_i, its ln xi_r, N_eff,sel r,
// flags, number of events, then (P > 0) the gradients of the first two.  xi = sum_r xi_r
// (the selection integral is a sum over injections), so
//   ln L = sum_r S_r - N ln xi,  grad = sum_r dS_r - N sum_r (xi_r / xi) d ln xi_r,
//   N_eff,sel = xi^2 / sum_r (xi_r^2 / N_eff,sel r)
// with N the events of all shards.  Flag bits 0 and 1 carry over; bit 3 (no injection
// weight) follows the merged xi; bit 2 (a shard's own selection cut) is dropped.
__host__ __device__ inline void merge_parts_point(int R, int K, int P, const double* parts, int k,
                                                  double* lnL_total, double* ln_xi, double* neff_sel,
                                                  int32_t* flags, double* grad_total) {
  const int W = 5 + 2 * P;
  double M = -INFINITY, ndet = 0.0;
  int fl = 0;
  bool dead = false;
  for (int r = 0; r < R; ++r) {
    const double* q = parts + ((size_t)r * K + k) * W;
    if (q[1] > M) M = q[1];
    ndet += q[4];
    fl |= (int)q[3];
    if (!(q[0] > -INFINITY && q[0] < INFINITY)) dead = true;
  }
  const bool fin = M > -INFINITY && M < INFINITY;
  double sw = 0.0, s2 = 0.0, se = 0.0;
  for (int r = 0; r < R; ++r) {
    const double* q = parts + ((size_t)r * K + k) * W;
    const double w = (fin && q[1] > -INFINITY) ? exp(q[1] - M) : 0.0;
    sw += w;
    if (q[2] > 0.0) s2 += w * w / q[2];
    se += q[0];
  }
  const double lx = (fin && sw > 0.0) ? M + log(sw) : -INFINITY;
  const int f = (fl & ~(4 | 8)) | (lx > -INFINITY ? 0 : 8);
  const bool bad = f != 0 || dead;
  lnL_total[k] = bad ? -INFINITY : se - ndet * lx;
  ln_xi[k] = lx;
  neff_sel[k] = s2 > 0.0 ? sw * sw / s2 : 0.0;
  flags[k] = f;
  if (P > 0 && grad_total) {
    for (int i = 0; i < P; ++i) {
      double ge = 0.0, gx = 0.0;
      for (int r = 0; r < R; ++r) {
        const double* q = parts + ((size_t)r * K + k) * W;
        const double w = (fin && q[1] > -INFINITY) ? exp(q[1] - M) : 0.0;
        ge += q[5 + i];
        gx += (sw > 0.0 ? w / sw : 0.0) * q[5 + P + i];
      }
      grad_total[(size_t)k * P + i] = bad ? 0.0 : ge - ndet * gx;
    }
  }
}
cudaError_t launch_merge_parts(int R, int K, int P, const double* parts, double* lnL_total, double* ln_xi,
                               double* neff_sel, int32_t* flags, double* grad_total, cudaStream_t s);

// the calling thread's message for gwc_last_error(NULL) (defined with the C ABI)
void set_thread_error(const std::string& msg);
cudaError_t launch_los_cell(const float* z, long long n, int nz, double zmax, int* cell, cudaStream_t s);

}  // namespace gwc
