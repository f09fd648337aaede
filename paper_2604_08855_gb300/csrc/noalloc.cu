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
#include <mutex>

#include "ctb_internal.cuh"

namespace ctb {

constexpr int kNoallocParts = 64;                   // contraction blocks (partial rows)
constexpr size_t kNoallocPartialDoubles = 1 << 20;  // 8 MB of FP64 partials
constexpr int kNoallocMaxDevices = 64;

// partial[part][l][b1][b2]; cleared at the start of every call
static __device__ __align__(256) double g_noalloc_partial[kNoallocPartialDoubles];
// identity slot table for rows in the l*l + l + m order (written at set-up)
static __device__ __align__(256) int g_noalloc_slot[(kLmaxCap + 1) * (kLmaxCap + 1)];

static __global__ void k_noalloc_identity(int* slot, int n) {
  for (int i = threadIdx.x; i < n; i += blockDim.x) slot[i] = i;
}

namespace {
struct DevScratch {
  bool ready = false;
  double* partial = nullptr;
  int* slot = nullptr;
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
  // (ell_max + 1) * nbins^2 must not exceed 16384: the fixed scratch holds 64 such blocks
  if (per_part * kNoallocParts > kNoallocPartialDoubles) return CTB_ERR_ARG;
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
      // set-up, once per device, with this device current
      void* p = nullptr;
      e = cudaGetSymbolAddress(&p, g_noalloc_partial);
      if (e != cudaSuccess) return CTB_ERR_CUDA;
      d.partial = static_cast<double*>(p);
      e = cudaGetSymbolAddress(&p, g_noalloc_slot);
      if (e != cudaSuccess) return CTB_ERR_CUDA;
      d.slot = static_cast<int*>(p);
      k_noalloc_identity<<<1, 256, 0, st>>>(d.slot, (kLmaxCap + 1) * (kLmaxCap + 1));
      ++g_launches;
      e = cudaGetLastError();
      if (e != cudaSuccess) return CTB_ERR_CUDA;
      d.ready = true;
    }
    sc = d;
  }
  // the partial sums are accumulated in place: clear the part this call uses
  e = cudaMemsetAsync(sc.partial, 0, per_part * kNoallocParts * sizeof(double), st);
  if (e != cudaSuccess) return CTB_ERR_CUDA;
  if (np > 0) {
    ContractArgs ca{};
    ca.M = alm;
    ca.wprim = w;
    ca.np = np;
    ca.nbins = nbins;
    ca.lmax = ell_max;
    ca.row = (ell_max + 1) * (ell_max + 1);
    ca.slot = sc.slot;
    ca.partial = sc.partial;
    ca.part0 = 0;
    e = launch_contract_fp32(ca, kNoallocParts, st);
    if (e != cudaSuccess) return CTB_ERR_CUDA;
  }
  e = launch_finalize(sc.partial, kNoallocParts, ell_max, nbins, zeta_out, false, st);
  if (e != cudaSuccess) return CTB_ERR_CUDA;
  return CTB_OK;
}
