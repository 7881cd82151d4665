// gwc_noalloc.cu -- gwc_sample_terms_noalloc: per-sample terms without any allocation.
//
// Some callers cannot allocate device memory at the moment they need an evaluation:
// code running while another component captures a CUDA graph (cudaMalloc is not
// allowed in a capturing stream), code inside a framework whose caching allocator owns
// the whole device budget, or callbacks that must not change the device's memory state.
// They cannot create a gwc_ctx (which owns device buffers).  This entry point evaluates
// the same per-sample terms as gwc_sample_terms from caller-owned device arrays and
// keeps its own scratch -- one Lambda point's constants and tables and the pixel-mean
// LOS row -- in a fixed file-scope device array, so a call allocates nothing.
//
// The scratch array is shared by every call in the process on a given device and keeps
// the last call's contents.  Each call first overwrites everything it later reads (the
// pixel slabs' partial sums, the pixel mean, the per-Lambda constants and the tables), so
// nothing needs to start at zero, but calls whose kernels overlap on the GPU (concurrent streams, or host threads
// issuing in parallel) race on the array and must be serialised by the caller.
#include <cmath>
#include <cstdint>
#include <cstring>
#include <mutex>
#include <string>

#include "../../include/gwc.h"
#include "gwc_kernels.h"

using namespace gwc;

namespace {

constexpr int MAX_NZ = 4096;      // LOS redshift nodes
constexpr int MAX_NX = 1024;      // nodes of the inversion table
constexpr int MAX_DEVICES = 64;
constexpr int PM_SLABS = 8;       // pixel slabs summed in parallel for the pixel mean

// scratch layout (bytes): LamF | LamD | per-Lambda tables | pixel mean (float) | (double)
// | the pixel slabs' partial sums (double, [PM_SLABS][n_z])
constexpr size_t OFF_LF = 0;
constexpr size_t OFF_LD = 512;
constexpr size_t OFF_TB = 1024;
constexpr size_t TB_BYTES = ((size_t)table_floats(MAX_NX) + 3) / 4 * 4 * sizeof(float);
constexpr size_t OFF_P32 = OFF_TB + (TB_BYTES + 255) / 256 * 256;
constexpr size_t OFF_P64 = OFF_P32 + (MAX_NZ * sizeof(float) + 255) / 256 * 256;
constexpr size_t OFF_PART = OFF_P64 + MAX_NZ * sizeof(double);
constexpr size_t SCRATCH_BYTES = OFF_PART + (size_t)PM_SLABS * MAX_NZ * sizeof(double);   // about 340 KB
static_assert(sizeof(LamF) <= OFF_LD - OFF_LF && sizeof(LamD) <= OFF_TB - OFF_LD, "scratch layout");

// Held by every device that loads the library, for the life of the process.
static __device__ __align__(256) unsigned char g_scratch[SCRATCH_BYTES];

std::mutex g_setup_mu;
unsigned char* g_scratch_ptr[MAX_DEVICES] = {nullptr};

// failures are reported through gwc_last_error(NULL), like the other context-free calls
gwc_status err(gwc_status s, const std::string& m) {
  set_thread_error(m);
  return s;
}

// Pixel mean of the LOS rows in two passes, every sum in FP64 and in a fixed order.  Pass
// 1: block (z tile, slab) has one thread per z node sum the slab's rows in row order, so
// PM_SLABS x n_z threads share the n_pix x n_z reads (coalesced along z).  Pass 2: one
// thread per z node adds the slabs' sums in slab order and divides by n_pix.
constexpr int PM_THREADS = 64;
__global__ void __launch_bounds__(PM_THREADS) k_pixel_mean_part(const float* __restrict__ los, int n_pix, int nz,
                                                                double* part) {
  const int j = blockIdx.x * PM_THREADS + threadIdx.x;
  if (j >= nz) return;
  const int slab = blockIdx.y;
  const int p0 = (int)((long long)n_pix * slab / PM_SLABS), p1 = (int)((long long)n_pix * (slab + 1) / PM_SLABS);
  double s = 0.0;
  for (int p = p0; p < p1; ++p) s += (double)__ldg(los + (size_t)p * nz + j);
  part[(size_t)slab * nz + j] = s;
}

__global__ void k_pixel_mean_combine(const double* __restrict__ part, int n_pix, int nz, float* p32, double* p64) {
  const int j = blockIdx.x * blockDim.x + threadIdx.x;
  if (j >= nz) return;
  double s = 0.0;
  for (int q = 0; q < PM_SLABS; ++q) s += part[(size_t)q * nz + j];
  s /= (double)n_pix;
  p64[j] = s;
  p32[j] = (float)s;
}

// One-time set-up on the current device: look up the device address of the scratch
// array (its host-side name is only a stand-in) and make sure the prologue's quadrature
// constants are on the device.
gwc_status setup(int dev, unsigned char** out) {
  std::lock_guard<std::mutex> g(g_setup_mu);
  if (g_scratch_ptr[dev]) {
    *out = g_scratch_ptr[dev];
    return GWC_OK;
  }
  void* p = nullptr;
  cudaError_t e = cudaGetSymbolAddress(&p, g_scratch);
  if (e != cudaSuccess) return err(GWC_E_CUDA, std::string("cudaGetSymbolAddress: ") + cudaGetErrorString(e));
  e = ensure_prologue_ready();
  if (e != cudaSuccess) return err(GWC_E_CUDA, std::string("constant upload: ") + cudaGetErrorString(e));
  g_scratch_ptr[dev] = static_cast<unsigned char*>(p);
  *out = g_scratch_ptr[dev];
  return GWC_OK;
}

}  // namespace

extern "C" gwc_status gwc_sample_terms_noalloc(const double* d_lambda, int64_t n_samples,
                                               const float* d_samples, const int32_t* d_pix,
                                               int64_t n_inj, const float* d_injections,
                                               int32_t n_pix, int32_t n_z, double z_max,
                                               const float* d_los, int32_t n_x_table, float* d_lnw,
                                               float* d_dlnw, double* d_c, void* stream) {
  if (n_z < 2 || n_z > MAX_NZ)
    return err(GWC_E_INVALID, "n_z must be in [2, " + std::to_string(MAX_NZ) + "] (scratch limit)");
  if (n_x_table < 16 || n_x_table > MAX_NX || n_x_table % 4 != 0)
    return err(GWC_E_INVALID, "n_x_table must be a multiple of 4 in [16, " + std::to_string(MAX_NX) +
                                  "] (scratch limit)");
  if (n_samples < 0 || n_inj < 0 || n_pix < 1 || !(z_max > 0.0))
    return err(GWC_E_INVALID, "bad sizes");
  if (!d_lambda || !d_los || !d_lnw || !d_c || (n_samples > 0 && (!d_samples || !d_pix)) ||
      (n_inj > 0 && !d_injections))
    return err(GWC_E_INVALID, "NULL device pointer");
  if ((reinterpret_cast<uintptr_t>(d_samples) | reinterpret_cast<uintptr_t>(d_injections)) & 15)
    return err(GWC_E_INVALID, "sample and injection arrays must be 16-byte aligned");
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return err(GWC_E_UNSUPPORTED, std::string("no CUDA device: ") + cudaGetErrorString(e));
  if (dev >= MAX_DEVICES) return err(GWC_E_UNSUPPORTED, "device index beyond the supported range");
  unsigned char* base = nullptr;
  gwc_status st = setup(dev, &base);
  if (st != GWC_OK) return st;
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  float* p32 = reinterpret_cast<float*>(base + OFF_P32);
  double* p64 = reinterpret_cast<double*>(base + OFF_P64);
  LamF* lf = reinterpret_cast<LamF*>(base + OFF_LF);
  LamD* ld = reinterpret_cast<LamD*>(base + OFF_LD);
  float* tables = reinterpret_cast<float*>(base + OFF_TB);

  double* part = reinterpret_cast<double*>(base + OFF_PART);
  k_pixel_mean_part<<<dim3((n_z + PM_THREADS - 1) / PM_THREADS, PM_SLABS), PM_THREADS, 0, s>>>(d_los, n_pix, n_z, part);
  e = cudaGetLastError();
  if (e == cudaSuccess) {
    k_pixel_mean_combine<<<(n_z + 255) / 256, 256, 0, s>>>(part, n_pix, n_z, p32, p64);
    e = cudaGetLastError();
  }
  if (e != cudaSuccess) return err(GWC_E_CUDA, std::string("pixel-mean launch: ") + cudaGetErrorString(e));
  ProArgs pa;
  pa.lam = d_lambda;
  pa.nx = n_x_table;
  pa.nz = n_z;
  pa.zmax = z_max;
  pa.pbar64 = p64;
  pa.lf = lf;
  pa.ld = ld;
  pa.tables = tables;
  pa.tstride = 0;
  pa.want_grad = 1;
  e = launch_prologue(pa, 1, s);
  if (e != cudaSuccess) return err(GWC_E_CUDA, std::string("prologue launch: ") + cudaGetErrorString(e));
  TermsArgs ta;
  ta.smp = reinterpret_cast<const float4*>(d_samples);
  ta.pix = d_pix;
  ta.inj = reinterpret_cast<const float4*>(d_injections);
  ta.los = d_los;
  ta.pbar32 = p32;
  ta.nz = n_z;
  ta.nx = n_x_table;
  ta.n_samples = n_samples;
  ta.n_total = n_samples + n_inj;
  ta.lf = lf;
  ta.ld = ld;
  ta.tables = tables;
  ta.lnw = d_lnw;
  ta.dlnw = d_dlnw;
  ta.c = d_c;
  ta.n_pix = n_pix;
  e = launch_sample_terms(ta, false, s);
  if (e != cudaSuccess) return err(GWC_E_CUDA, std::string("sample-terms launch: ") + cudaGetErrorString(e));
  return GWC_OK;
}
