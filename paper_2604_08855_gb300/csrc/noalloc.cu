// noalloc.cu -- zeta contraction that allocates no device memory.
//
// Some callers cannot allocate device memory when they call into this
// library: services that reserve the whole device up front in their own pool
// and hand out only fixed buffers, or loops with a latency budget in which an
// allocation (and its possible failure) is not acceptable.  This entry point
// serves them for one step of the path: given a_lm rows and primary weights
// already on the device, it runs the FP32 contraction kernel and the FP64
// normalisation with its per-block partial sums in a fixed, file-scope device
// array instead of allocated scratch.
//
// The array is a static __device__ object: every GPU that loads the library
// holds it until the process exits, and every call shares it (calls that
// overlap on the GPU race on it).  Host code must not use the array's name as
// a device address: the device address is taken with cudaGetSymbolAddress,
// once per device, with that device current, on the first call.
#include <algorithm>
#include <mutex>

#include "ctb_internal.cuh"

namespace ctb {

constexpr int kNoallocMinParts = 64;                // partial rows the size limit guarantees
constexpr size_t kNoallocPartialDoubles = 1 << 20;  // 8 MB of FP64 partials
constexpr int kNoallocMaxDevices = 64;

// partial[part][l][b1][b2]; the part a call uses is cleared at its start
static __device__ __align__(256) double g_noalloc_partial[kNoallocPartialDoubles];

// Identity slot table for rows in the l*l + l + m order.  It is constant-
// initialised in the module image, so no set-up kernel has to write it before
// the first contraction can read it.
struct IdentitySlots {
  int v[(kLmaxCap + 1) * (kLmaxCap + 1)];
  constexpr IdentitySlots() : v() {
    for (int i = 0; i < (kLmaxCap + 1) * (kLmaxCap + 1); ++i) v[i] = i;
  }
};
static __device__ __align__(256) IdentitySlots g_noalloc_slot = IdentitySlots();

namespace {
struct DevScratch {
  bool ready = false;
  double* partial = nullptr;
  int* slot = nullptr;
  int nsm = 0;
};
std::mutex g_noalloc_mu;
DevScratch g_noalloc_dev[kNoallocMaxDevices];
}  // namespace

}  // namespace ctb

using namespace ctb;

extern "C" int ctb_contract_noalloc(const float* alm, const float* w, int64_t np, int nbins, int ell_max,
                                    double* zeta_out, void* stream) {
  if (nbins < 1 || nbins > CTB_NBINS_CAP || ell_max < 0 || ell_max > CTB_LMAX_CAP) return CTB_ERR_ARG;
  if (np < 0) return CTB_ERR_ARG;
  if (!zeta_out || (np > 0 && (!alm || !w))) return CTB_ERR_ARG;
  const size_t per_part = (size_t)(ell_max + 1) * nbins * nbins;
  // (ell_max + 1) * nbins^2 must not exceed 16384: the fixed scratch holds at
  // least 64 partial blocks of that size
  if (per_part * kNoallocMinParts > kNoallocPartialDoubles) return CTB_ERR_ARG;
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return CTB_ERR_CUDA;
  if (dev < 0 || dev >= kNoallocMaxDevices) return CTB_ERR_ARG;
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  DevScratch sc;
  {
    std::lock_guard<std::mutex> lock(g_noalloc_mu);
    DevScratch& d = g_noalloc_dev[dev];
    if (!d.ready) {
      // set-up, once per device, with this device current: the device
      // addresses of the file-scope arrays and the SM count (no device work)
      void* p = nullptr;
      e = cudaGetSymbolAddress(&p, g_noalloc_partial);
      if (e != cudaSuccess) return CTB_ERR_CUDA;
      d.partial = static_cast<double*>(p);
      e = cudaGetSymbolAddress(&p, g_noalloc_slot);
      if (e != cudaSuccess) return CTB_ERR_CUDA;
      d.slot = static_cast<int*>(p);
      e = cudaDeviceGetAttribute(&d.nsm, cudaDevAttrMultiProcessorCount, dev);
      if (e != cudaSuccess || d.nsm < 1) return CTB_ERR_CUDA;
      d.ready = true;
    }
    sc = d;
  }
  // One partial row per contraction block: one wave of the kernel's resident
  // blocks (as ctb_compute runs it), as far as the fixed array holds them, so
  // that each block's FP32 run over its slice of the primaries stays short.
  const int row = (ell_max + 1) * (ell_max + 1);
  const int bps = contract_fp32_blocks_per_sm(nbins, ell_max, row, 0);
  if (bps < 1) return CTB_ERR_CUDA;
  const int nparts = (int)std::min<size_t>((size_t)bps * sc.nsm, kNoallocPartialDoubles / per_part);
  // the partial sums are accumulated in place: clear the part this call uses
  // (the finalisation reads exactly these nparts * per_part entries)
  e = cudaMemsetAsync(sc.partial, 0, per_part * nparts * sizeof(double), st);
  if (e != cudaSuccess) return CTB_ERR_CUDA;
  if (np > 0) {
    ContractArgs ca{};
    ca.M = alm;
    ca.wprim = w;
    ca.np = np;
    ca.nbins = nbins;
    ca.lmax = ell_max;
    ca.row = row;
    ca.slot = sc.slot;
    ca.partial = sc.partial;
    ca.part0 = 0;
    e = launch_contract_fp32(ca, nparts, st);
    if (e != cudaSuccess) return CTB_ERR_CUDA;
  }
  e = launch_finalize(sc.partial, nparts, ell_max, nbins, zeta_out, false, st);
  if (e != cudaSuccess) return CTB_ERR_CUDA;
  return CTB_OK;
}
