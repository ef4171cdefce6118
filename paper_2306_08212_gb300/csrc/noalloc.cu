// Singular values of a caller-provided device matrix without any device
// allocation.
//
// Some callers cannot allocate device memory at the moment they need this:
// code running inside a region where the allocator must not be touched (a
// custom memory manager that owns the whole device, an embedding runtime that
// forbids cudaMalloc/cudaFree after start-up, or a real-time loop where an
// allocation could stall).  They pass the input and the output; the scratch
// this computation needs (the working copy for the one-sided Jacobi sweeps, the
// column norms, the ordering and the grid-barrier words) lives in one
// file-scope __device__ array of fixed size, so nothing is allocated per call.
//
// The array is a host-side stand-in in host code, not a device address: its
// device address is taken once per device with cudaGetSymbolAddress (with that
// device current) during the first call on that device, and then handed to the
// kernels.  Do that first call before any stream capture begins.  Every GPU that
// loads this library holds the array (about 8.1 MB) until the process exits.
//
// All calls share the one array and it keeps the last call's contents: each
// call clears the words that must start at zero.  Calls whose GPU work overlaps
// (different streams, or different host threads on one device) race on the
// array and give wrong results; serialise them.  The Jacobi sweep itself is a
// cooperative launch issued, like every cooperative launch of this library, on
// one internal stream per device (created at the first such launch), ordered
// after the caller's stream with events; so it never waits on SMs held by a
// context's own cooperative kernels.
#include <cuda_runtime.h>

#include <mutex>

#include "../../include/ctm.h"
#include "ctm_internal.h"

namespace ctm {

constexpr long long kNoAllocMaxElems = 1ll << 20;  // rows * cols
constexpr int kNoAllocMaxSide = 4096;              // min(rows, cols)

// layout (doubles): X[kNoAllocMaxElems] | sig[kNoAllocMaxSide] |
//                   perm[kNoAllocMaxSide ints] | DevFlags
constexpr long long kSigOff = kNoAllocMaxElems;
constexpr long long kPermOff = kSigOff + kNoAllocMaxSide;
constexpr long long kFlagsOff = kPermOff + kNoAllocMaxSide / 2;
constexpr long long kScratchDoubles = kFlagsOff + 8;
static_assert(sizeof(DevFlags) <= 8 * sizeof(double), "DevFlags must fit its slot");

static __device__ __align__(256) double g_noalloc_scratch[kScratchDoubles];

namespace {

constexpr int kMaxDevices = 64;
std::mutex g_mu;
double* g_addr[kMaxDevices] = {};

// Device address of the scratch array on the current device (set up once).
int scratch_address(double** out) {
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= kMaxDevices) return CTM_ERR_CUDA;
  std::lock_guard<std::mutex> lock(g_mu);
  if (!g_addr[dev]) {
    void* p = nullptr;
    const cudaError_t e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
    if (e != cudaSuccess || !p) {
      cudaGetLastError();
      return CTM_ERR_CUDA;
    }
    g_addr[dev] = static_cast<double*>(p);
  }
  *out = g_addr[dev];
  return CTM_OK;
}

// s[r] = sig[perm[r]] / ||sig||  (one block; n <= kNoAllocMaxSide)
__global__ void sorted_unit_values_kernel(const double* __restrict__ sig,
                                          const int* __restrict__ perm, int n,
                                          double* __restrict__ s) {
  __shared__ double part[256];
  double acc = 0.0;
  for (int i = threadIdx.x; i < n; i += blockDim.x) acc = fma(sig[i], sig[i], acc);
  part[threadIdx.x] = acc;
  __syncthreads();
  for (int o = blockDim.x / 2; o > 0; o >>= 1) {
    if (threadIdx.x < o) part[threadIdx.x] += part[threadIdx.x + o];
    __syncthreads();
  }
  const double nrm = sqrt(part[0]);
  const double inv = nrm > 0.0 ? 1.0 / nrm : 0.0;
  for (int r = threadIdx.x; r < n; r += blockDim.x) s[r] = sig[perm[r]] * inv;
}

}  // namespace
}  // namespace ctm

extern "C" int ctm_singular_values_noalloc(const double* M, int rows, int cols, double* s,
                                           void* stream) {
  using namespace ctm;
  if (!M || !s || rows < 1 || cols < 1) return CTM_ERR_ARG;
  if ((long long)rows * cols > kNoAllocMaxElems || (rows < cols ? rows : cols) > kNoAllocMaxSide)
    return CTM_ERR_ARG;  // beyond the fixed scratch: rows*cols <= 2^20, min side <= 4096
  double* base = nullptr;
  const int rc = scratch_address(&base);
  if (rc != CTM_OK) return rc;
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  double* X = base;
  double* sig = base + kSigOff;
  int* perm = reinterpret_cast<int*>(base + kPermOff);
  DevFlags* flags = reinterpret_cast<DevFlags*>(base + kFlagsOff);
  // Jacobi on the columns of whichever orientation has fewer columns
  const bool cols_side = cols <= rows;
  const int nrows = cols_side ? rows : cols, ncols = cols_side ? cols : rows;
  if (cudaMemsetAsync(flags, 0, sizeof(DevFlags), st) != cudaSuccess) return CTM_ERR_CUDA;
  if (cols_side) {  // X column-major = M's columns
    LegMap m;
    m.n = 2;
    m.dim[0] = cols;
    m.stride[0] = 1;
    m.dim[1] = rows;
    m.stride[1] = cols;
    if (permute_f64(st, X, M, m) != cudaSuccess) return CTM_ERR_CUDA;
  } else {  // M row-major is M^T column-major
    if (cudaMemcpyAsync(X, M, sizeof(double) * (size_t)rows * cols, cudaMemcpyDeviceToDevice,
                        st) != cudaSuccess)
      return CTM_ERR_CUDA;
  }
  long long launches = 0;
  // serialize = true: the cooperative launch runs on the library's one
  // cooperative stream of this device, ordered after the work already issued on
  // `stream`, so it never contends with a context's own Jacobi launches for
  // co-residency (events only; no device memory is allocated)
  if (jacobi_batched(st, X, nrows, ncols, 1, 0, flags, 60, &launches, kValuesOnlyTol, true) != 0)
    return CTM_ERR_CUDA;
  if (column_norms_sorted(st, X, nrows, ncols, sig, perm) != cudaSuccess) return CTM_ERR_CUDA;
  sorted_unit_values_kernel<<<1, 256, 0, st>>>(sig, perm, ncols, s);
  if (cudaGetLastError() != cudaSuccess) return CTM_ERR_CUDA;
  DevFlags h;
  if (cudaMemcpyAsync(&h, flags, sizeof(DevFlags), cudaMemcpyDeviceToHost, st) != cudaSuccess ||
      cudaStreamSynchronize(st) != cudaSuccess)
    return CTM_ERR_CUDA;
  if (h.error) return CTM_ERR_CUDA;
  if (h.noconv) return CTM_ERR_NOCONV;
  return CTM_OK;
}
