// Adjoint of the truncated left singular vectors that define a projector
// (Sec. IV, Fig. 4a differentiated), in FP64.
//
// For M = U diag(s) Vt (thin, r = min(rows, cols), s descending) and the
// gradient gU of a loss with respect to the leading k columns of U:
//
//   gM = U [(F o (J - J^T)) diag(s)] Vt + (I - U U^T) gU diag(s_k)^-1 Vt_k
//
// with gU zero-padded to r columns, J = U^T gU and F_ij = E_ij / (E_ij^2 +
// eps s_0^4), E_ij = s_j^2 - s_i^2, F_ii = 0: the Lorentzian broadening of Liao,
// Liu, Wang & Xiang (PRX 9, 031041, 2019), relative to the largest singular
// value.  The second term (Townsend 2016) carries the part of gU outside the
// span of U; it vanishes when rows <= cols (U square).  S and Vt get no
// gradient: a projector v v^T uses the left vectors only.  Rank-deficient and
// degenerate inputs stay finite: with eps = 0 an exactly degenerate pair gets
// F_ij = 0, and a zero singular value the pseudo-inverse 0 in diag(s_k)^-1.
//
// Four FP64 leg-map GEMMs and two element-wise kernels; the GEMMs carry all the
// O(rows r^2 + rows r cols) work.
#include <cuda_runtime.h>

#include "../../include/ctm.h"
#include "ctm_internal.h"

namespace ctm {
namespace {

LegMap leg(int d, long long stride) {
  LegMap m;
  m.n = 1;
  m.dim[0] = d;
  m.stride[0] = stride;
  return m;
}

// X[i, j] = F_ij (J~[i, j] - J~[j, i]) s_j for the r x r core, J~ = J (r x k)
// zero-padded to r columns.
__global__ void adjoint_core_kernel(const double* __restrict__ J, const double* __restrict__ s,
                                    int r, int k, double eps, double* __restrict__ X) {
  const long long n = (long long)r * r;
  const double s0 = s[0];
  const double floor = eps * s0 * s0 * s0 * s0;
  for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < n;
       e += (long long)gridDim.x * blockDim.x) {
    const int i = (int)(e / r), j = (int)(e - (long long)i * r);
    double v = 0.0;
    if (i != j) {
      const double E = s[j] * s[j] - s[i] * s[i];
      const double den = E * E + floor;
      const double F = den > 0.0 ? E / den : 0.0;  // exactly degenerate, eps = 0: zero
      const double jij = j < k ? J[(long long)i * k + j] : 0.0;
      const double jji = i < k ? J[(long long)j * k + i] : 0.0;
      v = F * (jij - jji) * s[j];
    }
    X[e] = v;
  }
}

// T[row, j] += P[row, j] / s_j for j < k  (T: rows x r, P: rows x k); a zero
// singular value takes the pseudo-inverse 0.
__global__ void add_scaled_kernel(double* __restrict__ T, const double* __restrict__ P,
                                  const double* __restrict__ s, int rows, int r, int k) {
  const long long n = (long long)rows * k;
  for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < n;
       e += (long long)gridDim.x * blockDim.x) {
    const long long row = e / k;
    const int j = (int)(e - row * k);
    const double sj = s[j];
    if (sj > 0.0) T[row * r + j] += P[e] / sj;
  }
}

unsigned blocks_for(long long n) {
  long long b = (n + 255) / 256;
  if (b > 152 * 16) b = 152 * 16;
  return (unsigned)(b < 1 ? 1 : b);
}

}  // namespace
}  // namespace ctm

extern "C" int ctm_svd_left_adjoint(const double* U, const double* s, const double* Vt,
                                    const double* gU, int rows, int cols, int k, double eps,
                                    double* gM, void* stream) {
  using namespace ctm;
  const int r = rows < cols ? rows : cols;
  if (!U || !s || !Vt || !gU || !gM || rows < 1 || cols < 1 || k < 1 || k > r || !(eps >= 0.0))
    return CTM_ERR_ARG;
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  double *J = nullptr, *X = nullptr, *T = nullptr, *P = nullptr;
  const bool tall = rows > r;
  auto release = [&]() {
    if (J) cudaFreeAsync(J, st);
    if (X) cudaFreeAsync(X, st);
    if (T) cudaFreeAsync(T, st);
    if (P) cudaFreeAsync(P, st);
  };
  if (cudaMallocAsync(&J, sizeof(double) * (size_t)r * k, st) != cudaSuccess ||
      cudaMallocAsync(&X, sizeof(double) * (size_t)r * r, st) != cudaSuccess ||
      cudaMallocAsync(&T, sizeof(double) * (size_t)rows * r, st) != cudaSuccess ||
      (tall && cudaMallocAsync(&P, sizeof(double) * (size_t)rows * k, st) != cudaSuccess)) {
    cudaGetLastError();
    release();
    return CTM_ERR_OOM;
  }
  cudaError_t e = cudaSuccess;
  // J (r x k) = U^T gU
  e = gemm_f64(st, r, k, rows, 1.0, U, leg(r, 1), leg(rows, r), gU, leg(rows, k), leg(k, 1), 0.0,
               J, leg(r, k), leg(k, 1));
  if (e == cudaSuccess) {
    adjoint_core_kernel<<<blocks_for((long long)r * r), 256, 0, st>>>(J, s, r, k, eps, X);
    e = cudaGetLastError();
  }
  // T (rows x r) = U X
  if (e == cudaSuccess)
    e = gemm_f64(st, rows, r, r, 1.0, U, leg(rows, r), leg(r, 1), X, leg(r, r), leg(r, 1), 0.0, T,
                 leg(rows, r), leg(r, 1));
  if (tall && e == cudaSuccess) {
    // P (rows x k) = gU - U J, then T[:, :k] += P / s_k
    e = cudaMemcpyAsync(P, gU, sizeof(double) * (size_t)rows * k, cudaMemcpyDeviceToDevice, st);
    if (e == cudaSuccess)
      e = gemm_f64(st, rows, k, r, -1.0, U, leg(rows, r), leg(r, 1), J, leg(r, k), leg(k, 1), 1.0,
                   P, leg(rows, k), leg(k, 1));
    if (e == cudaSuccess) {
      add_scaled_kernel<<<blocks_for((long long)rows * k), 256, 0, st>>>(T, P, s, rows, r, k);
      e = cudaGetLastError();
    }
  }
  // gM (rows x cols) = T Vt
  if (e == cudaSuccess)
    e = gemm_f64(st, rows, cols, r, 1.0, T, leg(rows, r), leg(r, 1), Vt, leg(r, cols), leg(cols, 1),
                 0.0, gM, leg(rows, cols), leg(cols, 1));
  release();
  if (e != cudaSuccess) {
    cudaGetLastError();
    return CTM_ERR_CUDA;
  }
  return CTM_OK;
}
