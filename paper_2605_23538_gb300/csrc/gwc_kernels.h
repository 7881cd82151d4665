// gwc_kernels.h -- launch interface between the host API (gwc_api.cu) and the kernels.
#pragma once

#include <cstddef>
#include <cstdint>
#include <string>
#include <cuda_runtime.h>

#include "gwc_internal.cuh"

namespace gwc {

struct ProArgs {
  const double* lam;      // [K][13]
  int nx;                 // nodes of the inversion table
  int nz;                 // LOS grid nodes
  double zmax;
  const double* pbar64;   // [nz] pixel-averaged LOS prior (FP64)
  LamF* lf;               // [K]
  LamD* ld;               // [K]
  float* tables;          // [K][tstride]
  int tstride;
  int want_grad;
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
  float* partials;        // [K][n_items][PSTRIDE]
};

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
  const float* partials;
  int n_items;
  int P;
  const int32_t* ev_item0;  // [n_events + 1]
  int n_events;
  int inj_item0;
  const double* ev_n;       // [n_events] samples per event
  double n_draw;
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
};

cudaError_t set_gauss_legendre(const double* x, const double* w);
cudaError_t launch_prologue(const ProArgs& a, int K, cudaStream_t s);
constexpr int MAX_SLAB = 64;   // Lambda points per CTA tile at most
size_t fused_smem_bytes(int chunk, int slab, int group);
size_t fused_smem_max();
cudaError_t launch_fused(const FusedArgs& a, bool grad, bool kahan, bool bf16, int grid, cudaStream_t s);
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
  float* dlnw;      // [13][n_total] or nullptr
  double* c;        // [14]
};
cudaError_t launch_sample_terms(const TermsArgs& a, bool bf16, cudaStream_t s);
// the calling thread's message for gwc_last_error(NULL) (defined with the C ABI)
void set_thread_error(const std::string& msg);
cudaError_t launch_los_cell(const float* z, long long n, int nz, double zmax, int* cell, cudaStream_t s);

}  // namespace gwc
