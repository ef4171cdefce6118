// Internal declarations shared by the libctm translation units.
#pragma once

#include <cuda_runtime.h>

#include <cstdint>
#include <cstdio>
#include <string>
#include <vector>

namespace ctm {

constexpr int kMaxLegs = 12;

// A composite index over up to kMaxLegs sub-legs (row-major, last fastest);
// its memory offset is sum_l idx_l * stride_l.  Any leg permutation of a
// row-major tensor splits into an M-part and a K-part whose offsets add, so a
// GEMM operand can be read in any leg order without a transpose pass.
struct LegMap {
  int n = 0;
  int dim[kMaxLegs];
  long long stride[kMaxLegs];
  long long extent() const {
    long long e = 1;
    for (int i = 0; i < n; ++i) e *= dim[i];
    return e;
  }
};

// FP64 tensor view (device memory, row-major contiguous).
struct Ten {
  double* p = nullptr;
  int nd = 0;
  int dims[kMaxLegs] = {0};
  long long size() const {
    long long s = 1;
    for (int i = 0; i < nd; ++i) s *= dims[i];
    return s;
  }
  int rows_first(int nrow_legs) const {  // product of the first nrow_legs dims
    int r = 1;
    for (int i = 0; i < nrow_legs; ++i) r *= dims[i];
    return r;
  }
};

struct Status {
  int code = 0;
  std::string msg;
};

// Device-side error/status words of one context (zeroed at creation).
// The first block (barrier state and sweep maxima) is reset before every
// cooperative launch; the sticky words after it are cleared only by the host
// once it has read them.
struct DevFlags {
  unsigned int bar_count;
  unsigned int bar_gen;
  unsigned long long off_max[2];  // per-sweep max off-diagonal cosine (bits of a double >= 0)
  double fro2;                    // squared Frobenius norm of the Jacobi input
  int error;                      // sticky: a grid barrier timed out
  int noconv;                     // sticky: a Jacobi sweep cap was reached
  int bad;                        // sticky: a normalised tensor was zero or not finite
  int sweeps;                     // sweeps used by the last Jacobi launch
  int tc_timeout;                 // sticky: a tensor-core pipeline wait timed out (written
                                  // by those kernels only, never read by a kernel)
};
constexpr size_t kDevFlagsResetBytes = 32;  // offsetof(DevFlags, error)

// ---- kernels (gemm_f64.cu) ----
// C(m,n) = alpha * sum_k A(m,k) B(k,n) + beta * C(m,n), all FP64, every operand
// addressed through LegMaps.
cudaError_t gemm_f64(cudaStream_t s, long long M, long long N, long long K, double alpha,
                     const double* A, const LegMap& Am, const LegMap& Ak, const double* B,
                     const LegMap& Bk, const LegMap& Bn, double beta, double* C,
                     const LegMap& Cm, const LegMap& Cn);

// out[i] = in[map(i)] (gather permute), i over map.extent().
cudaError_t permute_f64(cudaStream_t s, double* out, const double* in, const LegMap& map);

// ---- linear algebra (linalg.cu) ----

// Fill x[0..n) with N(0,1) samples from a counter-based generator (SplitMix64
// hashing of (seed, index), Box-Muller); deterministic in (seed, n).
cudaError_t gaussian_fill(cudaStream_t s, double* x, long long n, unsigned long long seed);

// One-sided Jacobi (Hestenes) on the columns of X (nrows x ncols, column-major,
// leading dimension nrows), optionally accumulating the rotations in V
// (ncols x ncols column-major, initialised to the identity here).  On return
// the columns of X are mutually orthogonal.  Cooperative launch with a bounded
// grid barrier.  Returns 0, or CTM_ERR_NOCONV / CTM_ERR_CUDA style codes.
int jacobi_onesided(cudaStream_t s, double* X, int nrows, int ncols, double* V,
                    DevFlags* flags, int max_sweeps, long long* launches);

// nprob independent problems X + p * pstride in one launch (no accumulation).
// tol_override > 0 replaces the cosine tolerance sqrt(nrows) * eps; singular
// values alone converge quadratically in the cosines, so 1e-10 already gives
// them to FP64 accuracy.
// serialize: issue on the process-wide cooperative stream (see coop_stream).
// colver (values-only mode): nprob * (ncols + 1) ints of scratch for per-column
// step counters, which replace the grid barrier of every round-robin step; nullptr
// keeps the barrier per step (no scratch needed).
int jacobi_batched(cudaStream_t s, double* X, int nrows, int ncols, int nprob, long long pstride,
                   DevFlags* flags, int max_sweeps, long long* launches, double tol_override,
                   bool serialize, int* colver = nullptr);

// The stream on which every cooperative launch of this library runs (one per
// device, created on first use).
cudaStream_t coop_stream();

// Cooperative launch of fn on that stream, ordered after the work issued so far
// on s and before the work issued on s later (events).  t0 / t1 (optional) are
// recorded on the cooperative stream right before and after the kernel.
cudaError_t launch_cooperative(const void* fn, dim3 grid, dim3 block, void** args, size_t smem,
                               cudaStream_t s, cudaEvent_t t0 = nullptr,
                               cudaEvent_t t1 = nullptr);

// ---- fused CholeskyQR (cholqr.cu) ----
// Q (row-major rows x n) = an orthonormal basis of the columns of Y (row-major
// rows x n, not modified) by `passes` CholeskyQR passes, the first shifted when
// `shifted`, in one cooperative launch on the cooperative stream.  work holds
// cholqr_work_doubles(rows, n) doubles (not zeroed by the caller).  A barrier
// timeout sets *err_word; floored pivots of the shifted pass add to *floored.
// n <= 512.  Returns 0, -1 (arguments) or -3 (launch).
constexpr int kCholqrMaxN = 512;
constexpr int kCholqrMaxProb = 4;
size_t cholqr_work_doubles(int rows, int n, int nprob = 1);
// nprob (<= kCholqrMaxProb) independent problems of the same shape in one launch:
// they share the barriers and the latency-bound Cholesky steps.
// `passes` is the most a problem runs: a problem stops after an unshifted pass
// whose input was already well conditioned.  When flops_out is given, the
// launch adds the FP64 flops of the passes it ran to it (2 rows n^2 for the Gram
// and the substitution, n^3 / 3 for a Cholesky; rows n^2 for a pass that only
// rescales an orthonormal input).
int cholqr_fused_batch(cudaStream_t s, int nprob, const double* const* Y, double* const* Q,
                       int rows, int n, int passes, bool shifted, double* work, int* err_word,
                       int* floored, double* flops_out, unsigned long long seed,
                       long long* launches, cudaEvent_t t0 = nullptr, cudaEvent_t t1 = nullptr);
int cholqr_fused(cudaStream_t s, const double* Y, double* Q, int rows, int n, int passes,
                 bool shifted, double* work, int* err_word, int* floored, double* flops_out,
                 unsigned long long seed, long long* launches, cudaEvent_t t0 = nullptr,
                 cudaEvent_t t1 = nullptr);
// Diagnostics: after a launch on `work` (synchronises s), out[q * 16 + pass] =
// max |G' - I| and out[q * 16 + 8 + pass] = ||G' - I||_F^2 of problem q's scaled
// Gram in each pass it ran (zero for passes it skipped).
int cholqr_read_emax(cudaStream_t s, const double* work, int rows, int n, int nprob, double* out);
// Diagnostics under CTM_TRACE=3: summed ms of the last launch's phases, by tag
// (1 Gram, 2 reduction, 3 diagonal blocks, 4 panels, 5 trailing updates,
// 6 substitution).
unsigned long long* cq_stamps_buffer();
int cholqr_read_stamps(cudaStream_t s, double* ms_by_tag);
constexpr double kValuesOnlyTol = 1e-10;

// Preconditioner of the values-only Jacobi for nprob matrices C[p] (row-major
// n1 x n2, n2 <= n1): the same dataflow one-sided Jacobi run in FP32 on a copy,
// with the rotations accumulated into V; Vout[p] (row-major n2 x n2, FP64)
// receives V, orthonormal to FP32 accuracy.  X and V are FP32 scratch of
// nprob n1 n2 and nprob n2^2 floats, colver nprob (n2 + 1) ints.  Reaching the
// sweep cap is not an error.  Returns 0, -1 (arguments) or -3 (launch).
int jacobi_precondition_f32(cudaStream_t s, const double* const* C, int n1, int n2, int nprob,
                            float* X, float* V, double* const* Vout, DevFlags* flags,
                            int max_sweeps, double tol, double tiny_rel, int* colver,
                            long long* launches);

// Column norms of X (nrows x ncols col-major) into sig[ncols]; perm[r] = index of
// the r-th largest.  Single-block kernels.
cudaError_t column_norms_sorted(cudaStream_t s, const double* X, int nrows, int ncols,
                                double* sig, int* perm);

// U(row-major rows x k)[i, r] = X[perm[r]][i] / sig[perm[r]]  (normalise)   when V == nullptr
//                             = V[perm[r]][i]                 (accumulated) otherwise
// followed by the sign convention (largest-|entry| of each column positive).
cudaError_t gather_sorted_columns(cudaStream_t s, double* U, int rows, int k, const double* X,
                                  const double* V, const double* sig, const int* perm);

// x /= ||x||_F with a deterministic two-level reduction; scratch holds
// kNormScratch doubles (partials, then the norm at scratch[kNormScratch - 1]);
// sets *bad = 1 (device) if the norm is zero or not finite.
constexpr int kNormScratch = 305;
cudaError_t normalize_f64(cudaStream_t s, double* x, long long n, double* scratch, int* bad);

cudaError_t fill_identity(cudaStream_t s, double* x, int n);

// Adds the number of non-finite entries of x[0..n) to *out (device).
cudaError_t count_nonfinite(cudaStream_t s, const double* x, long long n, int* out);

// Blocked-Cholesky pieces (CholeskyQR).
cudaError_t chol_diag(cudaStream_t s, double* G, int lda, int j0, int jb, double* Linv,
                      double floor, int* floored, double tau, int* defmask);
cudaError_t replace_flagged(cudaStream_t s, double* Q, int rows, int n, int* defmask,
                            unsigned long long seed);
cudaError_t gram_scale(cudaStream_t s, double* G, int n, double* d, double shift_rel);
cudaError_t copy2d(cudaStream_t s, double* dst, long long dld, const double* src, long long sld,
                   int rows, int cols, const double* colscale, int c0);

}  // namespace ctm
