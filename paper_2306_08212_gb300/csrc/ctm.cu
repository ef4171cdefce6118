// Host orchestrator and C ABI of libctm: environment storage, the CTM moves in
// the standard and the reduced-sequential form, projector factorisations,
// observables.  Every arithmetic step runs in this library's CUDA kernels; the
// host only sequences launches and reads back scalars.
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <stdexcept>
#include <string>
#include <vector>

#include "../../include/ctm.h"
#include "ctm_internal.h"
#include "tc_gemm.h"

using namespace ctm;

namespace {

struct CtmError {
  int code;
  std::string msg;
};

[[noreturn]] void fail(int code, const std::string& msg) { throw CtmError{code, msg}; }

void ck(cudaError_t e, const char* what) {
  if (e != cudaSuccess) fail(CTM_ERR_CUDA, std::string(what) + ": " + cudaGetErrorString(e));
}

constexpr int kExactSvdMax = 1024;  // exact one-sided Jacobi up to this size
constexpr int kFastMinSide = 0;  // mixed precision: subspace iteration for every size
constexpr int kMinOversample = 16;  // randomized range finder: extra columns (at least)
constexpr int kMaxPowerIters = 40;  // randomized range finder: subspace iteration cap
constexpr int kCapturedPowerIters = 4;  // inside a stream capture (no host check possible)
constexpr double kSubspaceTol = 1e-12;  // RMS sine of the principal angles between sweeps
constexpr int kMaxSweeps = 60;
// kernel classes timed by ctm_profile_enable: 0 FP64 contraction, 1 TF32 and
// 2 BF16 tensor-core contraction, 3 Jacobi, 4 fused CholeskyQR
constexpr int kProfClasses = 5;
constexpr int kProfMaskAll = (1 << kProfClasses) - 1;

}  // namespace

struct ctm_ctx {
  cudaStream_t stream = nullptr;
  int d = 0, D = 0, chi = 0, chip = 0, precision = CTM_FP64;
  double* site[4][2] = {};  // rotated copies rot^r(A), rot^r(B): [r][x]
  double* dbl[4][2] = {};   // double-layer tensors a (fused legs), built on first use
  double* bnd = nullptr;    // boundary matrix (D x D)
  Ten env[2][4][2];         // [kind][k-1][x]: the current tensors
  double* buf[2][4][2][2] = {};  // two buffers per tensor
  int cur[2][4][2] = {};
  DevFlags* flags = nullptr;
  double* norm_scratch = nullptr;
  long long launches = 0;
  unsigned long long seed = 0x5eed;
  std::string err;
  std::vector<void*> owned;  // long-lived device allocations
  TcGemm* tc = nullptr;      // tensor-core GEMM state (mixed precision)
  struct ProfClass {
    std::vector<cudaEvent_t> ev;  // pairs (start, stop)
    size_t used = 0;
    long long count = 0;
    double ms = 0.0, flops = 0.0;
  };
  int prof_mask = 0;  // bit cls set: time that class
  bool prof_serial = false;  // calibration: one stream, eager launches (no graphs)
  ProfClass prof[kProfClasses];
  long long prof_seen[kProfClasses] = {};  // launches of each class (for sampling)
  struct CacheEntry {  // warm start of the mixed-precision subspace iteration
    double* p = nullptr;
    int rows = 0, k = 0;
  };
  CacheEntry cache[64];  // 0..47 split isometries, 48..55 standard, 56..63 reduced-env
  int* floored = nullptr;  // CholeskyQR pivots floored (device counter)
  double* cq_flops = nullptr;  // FP64 flops the CholeskyQR launches executed (device)
  double cq_flops_base = 0.0;  // its value when the profile counters were cleared
  // CUDA graphs of steady-state moves (mixed precision, reduced-sequential)
  struct GraphEvent {
    int cls;
    cudaEvent_t e0, e1;
    double flops;
  };
  cudaStream_t side[3] = {nullptr, nullptr, nullptr};  // for independent factorisations
  std::vector<cudaEvent_t> fork_events;
  size_t fork_next = 0;
  bool graphs_ok = true;
  bool capturing = false;
  int capture_dir = -1;
  bool warm[4] = {false, false, false, false};
  cudaGraphExec_t gexec[4] = {nullptr, nullptr, nullptr, nullptr};
  long long glaunches[4] = {0, 0, 0, 0};  // kernels in each graph
  std::vector<GraphEvent> gev[4];
};

namespace {

// ---------------------------------------------------------------------------
// Device memory
// ---------------------------------------------------------------------------
double* dalloc(ctm_ctx* c, long long n) {
  void* p = nullptr;
  if (n <= 0) n = 1;
  cudaError_t e = cudaMallocAsync(&p, (size_t)n * sizeof(double), c->stream);
  if (e != cudaSuccess) {
    cudaGetLastError();
    fail(CTM_ERR_OOM, "device allocation of " + std::to_string(n * 8) + " bytes failed");
  }
  return (double*)p;
}

void dfree(ctm_ctx* c, void* p) {
  if (p) cudaFreeAsync(p, c->stream);
}

double* owned_alloc(ctm_ctx* c, long long n) {
  void* p = nullptr;
  if (n <= 0) n = 1;
  if (cudaMalloc(&p, (size_t)n * sizeof(double)) != cudaSuccess) {
    cudaGetLastError();
    fail(CTM_ERR_OOM, "device allocation failed");
  }
  c->owned.push_back(p);
  return (double*)p;
}

// A temporary tensor freed (stream-ordered) when it leaves scope.
struct Tmp {
  ctm_ctx* c = nullptr;
  Ten t;
  Tmp() = default;
  Tmp(ctm_ctx* ctx, std::initializer_list<int> dims) : c(ctx) {
    t.nd = 0;
    for (int v : dims) t.dims[t.nd++] = v;
    t.p = dalloc(c, t.size());
  }
  Tmp(ctm_ctx* ctx, const int* dims, int nd) : c(ctx) {
    t.nd = nd;
    for (int i = 0; i < nd; ++i) t.dims[i] = dims[i];
    t.p = dalloc(c, t.size());
  }
  Tmp(const Tmp&) = delete;
  Tmp& operator=(const Tmp&) = delete;
  Tmp(Tmp&& o) noexcept : c(o.c), t(o.t) { o.t.p = nullptr; }
  Tmp& operator=(Tmp&& o) noexcept {
    if (this != &o) {
      release();
      c = o.c;
      t = o.t;
      o.t.p = nullptr;
    }
    return *this;
  }
  ~Tmp() { release(); }
  void release() {
    if (t.p && c) dfree(c, t.p);
    t.p = nullptr;
  }
  operator const Ten&() const { return t; }
};

Ten view(const Ten& t, std::initializer_list<int> dims) {
  Ten v;
  v.p = t.p;
  v.nd = 0;
  long long s = 1;
  for (int x : dims) {
    v.dims[v.nd++] = x;
    s *= x;
  }
  if (s != t.size()) fail(CTM_ERR_ARG, "internal: reshape size mismatch");
  return v;
}

// ---------------------------------------------------------------------------
// Optional per-class kernel timing (CUDA events on the context's stream)
// ---------------------------------------------------------------------------
struct ProfScope {
  ctm_ctx* c;
  int cls;
  size_t slot = 0;
  bool on;
  bool deferred;  // the callee records the two events around the kernel itself
  cudaEvent_t g0 = nullptr, g1 = nullptr;  // event pair owned by a graph being captured
  // When only the FP64 contractions are timed, one launch in kSampleF64 carries
  // events, to keep the overhead inside a timed region small.
  static constexpr int kSampleF64 = 8;
  ProfScope(ctm_ctx* ctx, int k, double flops, bool defer = false)
      : c(ctx), cls(k), on(((ctx->prof_mask >> k) & 1) != 0), deferred(defer) {
    // sampling only when the FP64 class is timed alone (the timed region), not
    // in the all-class breakdown
    if (on && cls == 0 && c->prof_mask == 1 && (c->prof_seen[0]++ % kSampleF64) != 0) on = false;
    if (c->capturing) {
      // launches of a timed class inside a captured move carry their own event
      // pair, recorded by every replay of the graph
      const bool sampled = on;
      on = false;
      if (sampled) {
        if (cudaEventCreate(&g0) != cudaSuccess || cudaEventCreate(&g1) != cudaSuccess)
          fail(CTM_ERR_CUDA, "event create");
        c->gev[c->capture_dir].push_back({cls, g0, g1, flops});
        if (!deferred) cudaEventRecordWithFlags(g0, c->stream, cudaEventRecordExternal);
      }
      return;
    }
    if (!on) return;
    auto& pc = c->prof[cls];
    if (pc.used + 2 > pc.ev.size()) {
      for (int i = 0; i < 64; ++i) {
        cudaEvent_t e;
        if (cudaEventCreate(&e) != cudaSuccess) fail(CTM_ERR_CUDA, "event create");
        pc.ev.push_back(e);
      }
    }
    slot = pc.used;
    pc.used += 2;
    pc.count += 1;
    pc.flops += flops;
    if (!deferred) cudaEventRecord(pc.ev[slot], c->stream);
  }
  cudaEvent_t ev0() const { return g0 ? g0 : (on ? c->prof[cls].ev[slot] : nullptr); }
  cudaEvent_t ev1() const { return g1 ? g1 : (on ? c->prof[cls].ev[slot + 1] : nullptr); }
  ~ProfScope() {
    if (g1 && !deferred) cudaEventRecordWithFlags(g1, c->stream, cudaEventRecordExternal);
    if (on && !deferred) cudaEventRecord(c->prof[cls].ev[slot + 1], c->stream);
  }
};

void prof_collect(ctm_ctx* c) {
  cudaStreamSynchronize(c->stream);
  for (auto& pc : c->prof) {
    for (size_t i = 0; i + 1 < pc.used; i += 2) {
      float ms = 0.f;
      if (cudaEventElapsedTime(&ms, pc.ev[i], pc.ev[i + 1]) == cudaSuccess) pc.ms += ms;
    }
    pc.used = 0;
  }
  cudaGetLastError();
}

// ---------------------------------------------------------------------------
// Pairwise contraction "labelsA,labelsB->labelsOut" on FP64 tensors
// ---------------------------------------------------------------------------
struct Spec {
  std::string a, b, o;
};

Spec parse(const char* spec) {
  Spec s;
  const char* comma = std::strchr(spec, ',');
  const char* arrow = std::strstr(spec, "->");
  if (!comma || !arrow || arrow < comma) fail(CTM_ERR_ARG, std::string("internal: bad spec ") + spec);
  s.a.assign(spec, comma);
  s.b.assign(comma + 1, arrow);
  s.o.assign(arrow + 2);
  return s;
}

void strides_of(const Ten& t, long long* st) {
  long long s = 1;
  for (int i = t.nd - 1; i >= 0; --i) {
    st[i] = s;
    s *= t.dims[i];
  }
}

struct Plan {
  long long M = 1, N = 1, K = 1;
  LegMap Am, Ak, Bk, Bn, Cm, Cn;
  int out_dims[kMaxLegs];
  int out_nd = 0;
};

void push(LegMap& m, int dim, long long stride) {
  if (m.n >= kMaxLegs) fail(CTM_ERR_ARG, "internal: too many legs");
  m.dim[m.n] = dim;
  m.stride[m.n] = stride;
  ++m.n;
}

// Merge neighbouring sub-legs that are contiguous in both maps (fewer div/mods).
void merge_pair(LegMap& x, LegMap& y) {
  int w = 0;
  for (int i = 0; i < x.n; ++i) {
    if (w > 0 && x.stride[w - 1] == (long long)x.dim[i] * x.stride[i] &&
        y.stride[w - 1] == (long long)y.dim[i] * y.stride[i]) {
      x.dim[w - 1] *= x.dim[i];
      x.stride[w - 1] = x.stride[i];
      y.dim[w - 1] = x.dim[w - 1];
      y.stride[w - 1] = y.stride[i];
    } else {
      x.dim[w] = x.dim[i];
      x.stride[w] = x.stride[i];
      y.dim[w] = y.dim[i];
      y.stride[w] = y.stride[i];
      ++w;
    }
  }
  x.n = y.n = w;
}

Plan make_plan(const Spec& s, const Ten& A, const Ten& B) {
  if ((int)s.a.size() != A.nd || (int)s.b.size() != B.nd)
    fail(CTM_ERR_ARG, "internal: spec rank mismatch " + s.a + "," + s.b);
  long long sa[kMaxLegs], sb[kMaxLegs];
  strides_of(A, sa);
  strides_of(B, sb);
  auto dim_of = [&](char ch) -> int {
    size_t i = s.a.find(ch);
    if (i != std::string::npos) return A.dims[i];
    i = s.b.find(ch);
    if (i != std::string::npos) return B.dims[i];
    fail(CTM_ERR_ARG, std::string("internal: unknown label ") + ch);
  };
  Plan p;
  p.out_nd = (int)s.o.size();
  long long so[kMaxLegs];
  for (int i = 0; i < p.out_nd; ++i) p.out_dims[i] = dim_of(s.o[i]);
  {
    long long st = 1;
    for (int i = p.out_nd - 1; i >= 0; --i) {
      so[i] = st;
      st *= p.out_dims[i];
    }
  }
  for (int i = 0; i < p.out_nd; ++i) {
    const char ch = s.o[i];
    const size_t ia = s.a.find(ch), ib = s.b.find(ch);
    if (ia != std::string::npos && ib != std::string::npos)
      fail(CTM_ERR_ARG, "internal: batch labels are not supported");
    if (ia != std::string::npos) {
      push(p.Am, A.dims[ia], sa[ia]);
      push(p.Cm, A.dims[ia], so[i]);
      p.M *= A.dims[ia];
    } else if (ib != std::string::npos) {
      push(p.Bn, B.dims[ib], sb[ib]);
      push(p.Cn, B.dims[ib], so[i]);
      p.N *= B.dims[ib];
    } else {
      fail(CTM_ERR_ARG, "internal: output label not in inputs");
    }
  }
  for (int i = 0; i < A.nd; ++i) {
    const char ch = s.a[i];
    if (s.o.find(ch) != std::string::npos) continue;
    const size_t ib = s.b.find(ch);
    if (ib == std::string::npos) fail(CTM_ERR_ARG, "internal: traces are not supported");
    if (A.dims[i] != B.dims[ib])
      fail(CTM_ERR_ARG, std::string("internal: dim mismatch on label ") + ch + " in " + s.a +
                            "," + s.b);
    push(p.Ak, A.dims[i], sa[i]);
    push(p.Bk, B.dims[ib], sb[ib]);
    p.K *= A.dims[i];
  }
  for (int i = 0; i < B.nd; ++i)
    if (s.o.find(s.b[i]) == std::string::npos && s.a.find(s.b[i]) == std::string::npos)
      fail(CTM_ERR_ARG, "internal: traces are not supported");
  merge_pair(p.Am, p.Cm);
  merge_pair(p.Bn, p.Cn);
  merge_pair(p.Ak, p.Bk);
  return p;
}

// CTM_CHECK=1: after each contraction / factorisation, synchronise and report
// the first step that produced a non-finite value (debugging aid).
bool check_on() {
  static int on = -1;
  if (on < 0) {
    const char* e = std::getenv("CTM_CHECK");
    on = (e && *e && *e != '0') ? 1 : 0;
  }
  return on == 1;
}

void check_finite(ctm_ctx* c, const Ten& t, const char* what) {
  if (!check_on()) return;
  int* d = c->floored + 1;
  ck(cudaMemsetAsync(d, 0, sizeof(int), c->stream), "memset");
  ck(count_nonfinite(c->stream, t.p, t.size(), d), "count");
  int h = 0;
  ck(cudaMemcpyAsync(&h, d, sizeof(int), cudaMemcpyDeviceToHost, c->stream), "d2h");
  ck(cudaStreamSynchronize(c->stream), "sync");
  if (h) {
    std::fprintf(stderr, "[ctm] non-finite after %s (%d entries, dims", what, h);
    for (int i = 0; i < t.nd; ++i) std::fprintf(stderr, " %d", t.dims[i]);
    std::fprintf(stderr, ")\n");
  }
}

// C = A . B per the spec, FP64 always (factorisation-side and observables).
Tmp ein64(ctm_ctx* c, const char* spec, const Ten& A, const Ten& B) {
  Plan p = make_plan(parse(spec), A, B);
  Tmp C(c, p.out_dims, p.out_nd);
  {
    ProfScope ps(c, 0, 2.0 * p.M * p.N * p.K);
    ck(gemm_f64(c->stream, p.M, p.N, p.K, 1.0, A.p, p.Am, p.Ak, B.p, p.Bk, p.Bn, 0.0, C.t.p,
                p.Cm, p.Cn),
       spec);
  }
  ++c->launches;
  return C;
}

// Absorption / renormalisation contraction in the context's precision.
Tmp ein(ctm_ctx* c, const char* spec, const Ten& A, const Ten& B) {
  if (c->precision == CTM_FP64) return ein64(c, spec, A, B);
  Plan p = make_plan(parse(spec), A, B);
  Tmp C(c, p.out_dims, p.out_nd);
  ProfScope ps(c, c->precision == CTM_TF32 ? 1 : 2, 2.0 * p.M * p.N * p.K, true);
  int rc = tc_contract(c->tc, c->stream, c->precision, p.M, p.N, p.K, A.p, p.Am, p.Ak, B.p,
                       p.Bk, p.Bn, C.t.p, p.Cm, p.Cn, &c->launches, &c->flags->tc_timeout, ps.ev0(),
                       ps.ev1());
  if (rc != 0)
    fail(CTM_ERR_CUDA, std::string("tensor-core contraction failed (") + std::to_string(rc) + ", " +
                           cudaGetErrorString(cudaGetLastError()) + "): " + spec);
  check_finite(c, C.t, spec);
  return C;
}

// ---------------------------------------------------------------------------
// Factorisations (FP64)
// ---------------------------------------------------------------------------
void jacobi(ctm_ctx* c, double* X, int nrows, int ncols, double* V) {
  ProfScope ps(c, 3, 0.0);
  int rc = jacobi_onesided(c->stream, X, nrows, ncols, V, c->flags, kMaxSweeps, &c->launches);
  if (rc != 0) fail(CTM_ERR_CUDA, "Jacobi launch failed");
}

Tmp identity(ctm_ctx* c, int n) {
  Tmp I(c, {n, n});
  ck(fill_identity(c->stream, I.t.p, n), "identity");
  ++c->launches;
  return I;
}

// Orthonormal, sign-fixed, descending-ordered columns of X (col-major nrows x ncols)
// after Jacobi: U (row-major nrows x k) = X[:, perm[:k]] / sigma.
Tmp sorted_unit_columns(ctm_ctx* c, double* X, int nrows, int ncols, int k) {
  Tmp sig(c, {ncols});
  int* perm = (int*)dalloc(c, (ncols + 1) / 2 + 1);
  ck(column_norms_sorted(c->stream, X, nrows, ncols, sig.t.p, perm), "column norms");
  Tmp U(c, {nrows, k});
  ck(gather_sorted_columns(c->stream, U.t.p, nrows, k, X, nullptr, sig.t.p, perm), "gather");
  c->launches += 3;
  dfree(c, perm);
  return U;
}

// Leading k left singular vectors of the row-major matrix M (rows x cols):
// U (row-major rows x k).  Exact one-sided Jacobi when the smaller side is at
// most kExactSvdMax, else a randomized subspace iteration (Halko, Martinsson &
// Tropp, SIAM Rev. 53, 217 (2011)) run until its leading-k subspace stops
// moving, with a Jacobi SVD of the projected problem.  path: 0 = that choice,
// 1 = exact, 2 = randomized (test hook).
enum SvdPath { kSvdAuto = 0, kSvdExact = 1, kSvdRandomized = 2 };
Tmp left_svd_impl(ctm_ctx* c, const double* M, int rows, int cols, int k, int path = kSvdAuto,
                  int slot = -1);


// CTM_TRACE (any non-zero level) prints every factorisation (shape, path, time,
// Jacobi sweeps of the last launch), the CholeskyQR orthogonality per pass and
// the sweeps of the corner spectra to stderr, synchronising around each call;
// level 2 adds every contraction (tc_gemm.cu), level 3 the CholeskyQR phase
// times (cholqr.cu).
bool trace_on() {
  static int on = -1;
  if (on < 0) {
    const char* e = std::getenv("CTM_TRACE");
    on = (e && *e && *e != '0') ? 1 : 0;
  }
  return on == 1;
}

Tmp left_svd(ctm_ctx* c, const double* M, int rows, int cols, int k, int slot = -1) {
  if (!trace_on()) return left_svd_impl(c, M, rows, cols, k, kSvdAuto, slot);
  ck(cudaStreamSynchronize(c->stream), "sync");
  cudaEvent_t e0, e1;
  cudaEventCreate(&e0);
  cudaEventCreate(&e1);
  cudaEventRecord(e0, c->stream);
  Tmp U = left_svd_impl(c, M, rows, cols, k, kSvdAuto, slot);
  cudaEventRecord(e1, c->stream);
  ck(cudaStreamSynchronize(c->stream), "sync");
  float ms = 0.f;
  cudaEventElapsedTime(&ms, e0, e1);
  DevFlags h;
  cudaMemcpy(&h, c->flags, sizeof h, cudaMemcpyDeviceToHost);
  const char* path = k >= rows ? "identity" : (std::min(rows, cols) <= kExactSvdMax ? "exact" : "randomized");
  std::fprintf(stderr, "[ctm] svd %dx%d k=%d %s %.3f ms sweeps(last)=%d err=%d noconv=%d\n", rows,
               cols, k, path, ms, h.sweeps, h.error, h.noconv);
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  return U;
}

// Under CTM_TRACE (outside captures): the orthogonality error max |G' - I| that
// each pass of a fused CholeskyQR launch started from.
void trace_cholqr(ctm_ctx* c, const double* work, int rows, int n, int nprob, int passes) {
  if (!trace_on() || c->capturing) return;
  double e[16 * kCholqrMaxProb];
  if (cholqr_read_emax(c->stream, work, rows, n, nprob, e) != 0) return;
  std::fprintf(stderr, "[ctm] cholqr %dx%d x%d passes=%d max|G'-I|/||G'-I||_F:", rows, n, nprob,
               passes);
  for (int q = 0; q < nprob; ++q) {
    std::fprintf(stderr, " [");
    for (int p = 0; p < passes; ++p)
      std::fprintf(stderr, p ? " %.1e/%.1e" : "%.1e/%.1e", e[16 * q + p],
                   std::sqrt(e[16 * q + 8 + p]));
    std::fprintf(stderr, "]");
  }
  std::fprintf(stderr, "\n");
  double ph[8];
  if (cholqr_read_stamps(c->stream, ph) == 0)
    std::fprintf(stderr,
                 "[ctm] cholqr phases ms: gram %.3f reduce %.3f diag %.3f panel %.3f trailing %.3f "
                 "subst %.3f\n",
                 ph[1], ph[2], ph[3], ph[4], ph[5], ph[6]);
}

// Root-mean-square sine of the principal angles between the spans of the
// leading k columns of Uold and Unew (row-major rows x ld, orthonormal columns):
// ||Unew_k - Uold_k (Uold_k^T Unew_k)||_F / sqrt(k).  Synchronises the stream.
double subspace_change(ctm_ctx* c, const double* Uold, const double* Unew, int rows, int ld,
                       int k);

// Randomized subspace iteration run to convergence (defined with the
// CholeskyQR it orthonormalises with).
Tmp left_svd_subspace(ctm_ctx* c, const double* M, int rows, int cols, int k, int slot);

Tmp left_svd_impl(ctm_ctx* c, const double* M, int rows, int cols, int k, int path, int slot) {
  if (k >= rows) return identity(c, rows);
  if (k > std::min(rows, cols)) fail(CTM_ERR_ARG, "truncation rank exceeds the matrix rank bound");
  const bool exact = path == kSvdExact || (path == kSvdAuto && std::min(rows, cols) <= kExactSvdMax);
  if (exact) {
    if (cols <= rows) {
      // X = M column-major (transpose copy), Jacobi on its cols columns
      Tmp X(c, {cols, rows});
      LegMap m;
      push(m, cols, 1);
      push(m, rows, cols);
      ck(permute_f64(c->stream, X.t.p, M, m), "transpose");
      ++c->launches;
      jacobi(c, X.t.p, rows, cols, nullptr);
      return sorted_unit_columns(c, X.t.p, rows, cols, k);
    }
    // X = M^T column-major is M row-major; accumulate V (rows x rows)
    Tmp X(c, {rows, cols});
    ck(cudaMemcpyAsync(X.t.p, M, sizeof(double) * (size_t)rows * cols, cudaMemcpyDeviceToDevice,
                       c->stream),
       "copy");
    Tmp V(c, {rows, rows});
    jacobi(c, X.t.p, cols, rows, V.t.p);
    Tmp sig(c, {rows});
    int* perm = (int*)dalloc(c, (rows + 1) / 2 + 1);
    ck(column_norms_sorted(c->stream, X.t.p, cols, rows, sig.t.p, perm), "norms");
    Tmp U(c, {rows, k});
    ck(gather_sorted_columns(c->stream, U.t.p, rows, k, nullptr, V.t.p, sig.t.p, perm), "gather");
    c->launches += 3;
    dfree(c, perm);
    return U;
  }
  return left_svd_subspace(c, M, rows, cols, k, slot);
}

double subspace_change(ctm_ctx* c, const double* Uold, const double* Unew, int rows, int ld,
                       int k) {
  // S = Uold_k^T Unew_k (k x k)
  Tmp S(c, {k, k});
  {
    LegMap Am, Ak, Bk, Bn, Cm, Cn;
    push(Am, k, 1);
    push(Ak, rows, ld);
    push(Bk, rows, ld);
    push(Bn, k, 1);
    push(Cm, k, k);
    push(Cn, k, 1);
    ProfScope ps(c, 0, 2.0 * k * k * rows);
    ck(gemm_f64(c->stream, k, k, rows, 1.0, Uold, Am, Ak, Unew, Bk, Bn, 0.0, S.t.p, Cm, Cn),
       "U^T U");
    ++c->launches;
  }
  // R = Unew_k - Uold_k S
  Tmp R(c, {rows, k});
  {
    LegMap m;
    push(m, rows, ld);
    push(m, k, 1);
    ck(permute_f64(c->stream, R.t.p, Unew, m), "copy");
    ++c->launches;
    LegMap Am, Ak, Bk, Bn, Cm, Cn;
    push(Am, rows, ld);
    push(Ak, k, 1);
    push(Bk, k, k);
    push(Bn, k, 1);
    push(Cm, rows, k);
    push(Cn, k, 1);
    ProfScope ps(c, 0, 2.0 * k * k * rows);
    ck(gemm_f64(c->stream, rows, k, k, -1.0, Uold, Am, Ak, S.t.p, Bk, Bn, 1.0, R.t.p, Cm, Cn),
       "R");
    ++c->launches;
  }
  Tmp nn = ein64(c, "ij,ij->", R.t, R.t);
  double v = 0.0;
  ck(cudaMemcpyAsync(&v, nn.t.p, sizeof(double), cudaMemcpyDeviceToHost, c->stream), "d2h");
  ck(cudaStreamSynchronize(c->stream), "sync");
  return std::sqrt(std::max(v, 0.0) / k);
}

// ---------------------------------------------------------------------------
// Mixed-precision factorisation path
// ---------------------------------------------------------------------------
LegMap lm1(int d0, long long s0) {
  LegMap m;
  push(m, d0, s0);
  return m;
}

void gemm64(ctm_ctx* c, long long M, long long N, long long K, double alpha, const double* A,
            const LegMap& Am, const LegMap& Ak, const double* B, const LegMap& Bk,
            const LegMap& Bn, double beta, double* C, const LegMap& Cm, const LegMap& Cn) {
  ProfScope ps(c, 0, 2.0 * M * N * K);
  ck(gemm_f64(c->stream, M, N, K, alpha, A, Am, Ak, B, Bk, Bn, beta, C, Cm, Cn), "gemm");
  ++c->launches;
}

// Sketch products of the subspace iteration in the context's precision.
void gemm_mixed(ctm_ctx* c, long long M, long long N, long long K, const double* A,
                const LegMap& Am, const LegMap& Ak, const double* B, const LegMap& Bk,
                const LegMap& Bn, double* C, const LegMap& Cm, const LegMap& Cn) {
  if (c->precision == CTM_FP64) {
    gemm64(c, M, N, K, 1.0, A, Am, Ak, B, Bk, Bn, 0.0, C, Cm, Cn);
    return;
  }
  ProfScope ps(c, c->precision == CTM_TF32 ? 1 : 2, 2.0 * M * N * K, true);
  if (tc_contract(c->tc, c->stream, c->precision, M, N, K, A, Am, Ak, B, Bk, Bn, C, Cm, Cn,
                  &c->launches, &c->flags->tc_timeout, ps.ev0(), ps.ev1()) != 0)
    fail(CTM_ERR_CUDA, "tensor-core sketch product failed");
}

// Orthonormal basis Q (row-major rows x n) of the columns of Y, whose entry
// (i, j) sits at Y[i * ys_r + j * ys_c], by `passes` CholeskyQR passes in FP64:
// G = Q^T Q, column scaling D, G' = D^-1 G D^-1 (+ shift on the first pass),
// blocked Cholesky G' = L L^T (32-wide panels, updates as GEMMs), Q <- Q D^-1 L^-T.
Tmp cholqr_chain(ctm_ctx* c, const double* Y, long long ys_r, long long ys_c, int rows, int n,
                 int passes);

Tmp cholqr(ctm_ctx* c, const double* Y, long long ys_r, long long ys_c, int rows, int n,
           int passes) {
  if (n > kCholqrMaxN || ys_r != n || ys_c != 1 || rows < n)
    return cholqr_chain(c, Y, ys_r, ys_c, rows, n, passes);
  Tmp Q(c, {rows, n});
  Tmp W(c, {(int)cholqr_work_doubles(rows, n)});
  {
    // the timing events bracket the kernel on the cooperative stream; the kernel
    // adds the flops of the passes it ran to c->cq_flops
    ProfScope ps(c, 4, 0.0, true);
    const int rc = cholqr_fused(c->stream, Y, Q.t.p, rows, n, passes, true, W.t.p,
                                &c->flags->error, c->floored, c->cq_flops, c->seed,
                                &c->launches, ps.ev0(), ps.ev1());
    c->seed += passes;
    if (rc != 0) fail(CTM_ERR_CUDA, "fused CholeskyQR launch failed");
  }
  trace_cholqr(c, W.t.p, rows, n, 1, passes);
  check_finite(c, Q.t, "cholqr");
  return Q;
}

// The same passes as a chain of separate launches (blocked Cholesky with 32-wide
// panels, updates as FP64 GEMMs); for n above the fused kernel's limit.
Tmp cholqr_chain(ctm_ctx* c, const double* Y, long long ys_r, long long ys_c, int rows, int n,
                 int passes) {
  constexpr int NB = 32;
  const int nblk = (n + NB - 1) / NB;
  Tmp Q(c, {rows, n});
  {
    LegMap m;
    push(m, rows, ys_r);
    push(m, n, ys_c);
    ck(permute_f64(c->stream, Q.t.p, Y, m), "copy");
    ++c->launches;
  }
  Tmp Qn(c, {rows, n}), G(c, {n, n}), d(c, {n}), Linv(c, {nblk * NB * NB}), P(c, {n, NB}),
      T(c, {rows, NB});
  int* defmask = (int*)dalloc(c, (n + 1) / 2 + 1);
  ck(cudaMemsetAsync(defmask, 0, sizeof(int) * n, c->stream), "mask");
  const double u = 1.1102230246251565e-16;
  for (int pass = 0; pass < passes; ++pass) {
    // G = Q^T Q
    gemm64(c, n, n, rows, 1.0, Q.t.p, lm1(n, 1), lm1(rows, n), Q.t.p, lm1(rows, n), lm1(n, 1), 0.0,
           G.t.p, lm1(n, n), lm1(n, 1));
    const double shift = pass == 0 ? 11.0 * ((double)rows * n + (double)n * (n + 1)) * u : 0.0;
    ck(gram_scale(c->stream, G.t.p, n, d.t.p, shift), "gram scale");
    ++c->launches;
    for (int j0 = 0; j0 < n; j0 += NB) {
      const int jb = std::min(NB, n - j0);
      double* Lj = Linv.t.p + (long long)(j0 / NB) * NB * NB;
      // unshifted passes: a pivot below 1e-12 (of the unit scaled diagonal) marks a
      // column that lies in the span of the earlier ones; it is replaced below
      ck(chol_diag(c->stream, G.t.p, n, j0, jb, Lj, 1e-28, c->floored, pass == 0 ? 0.0 : 1e-12,
                   pass == 0 ? nullptr : defmask),
         "chol diag");
      ++c->launches;
      const int m2 = n - j0 - jb;
      if (m2 > 0) {
        double* A21 = G.t.p + (long long)(j0 + jb) * n + j0;
        gemm64(c, m2, jb, jb, 1.0, A21, lm1(m2, n), lm1(jb, 1), Lj, lm1(jb, 1), lm1(jb, NB), 0.0,
               P.t.p, lm1(m2, NB), lm1(jb, 1));
        ck(copy2d(c->stream, A21, n, P.t.p, NB, m2, jb, nullptr, 0), "copy");
        ++c->launches;
        double* G22 = G.t.p + (long long)(j0 + jb) * n + j0 + jb;
        gemm64(c, m2, m2, jb, -1.0, P.t.p, lm1(m2, NB), lm1(jb, 1), P.t.p, lm1(jb, 1),
               lm1(m2, NB), 1.0, G22, lm1(m2, n), lm1(m2, 1));
      }
    }
    for (int j0 = 0; j0 < n; j0 += NB) {
      const int jb = std::min(NB, n - j0);
      ck(copy2d(c->stream, T.t.p, NB, Q.t.p + j0, n, rows, jb, d.t.p, j0), "copy");
      ++c->launches;
      if (j0 > 0)
        gemm64(c, rows, jb, j0, -1.0, Qn.t.p, lm1(rows, n), lm1(j0, 1), G.t.p + (long long)j0 * n,
               lm1(j0, 1), lm1(jb, n), 1.0, T.t.p, lm1(rows, NB), lm1(jb, 1));
      const double* Lj = Linv.t.p + (long long)(j0 / NB) * NB * NB;
      gemm64(c, rows, jb, jb, 1.0, T.t.p, lm1(rows, NB), lm1(jb, 1), Lj, lm1(jb, 1), lm1(jb, NB),
             0.0, Qn.t.p + j0, lm1(rows, n), lm1(jb, 1));
    }
    std::swap(Q, Qn);
    if (pass > 0 && pass + 1 < passes) {  // rank deficiency: random columns, orthonormalised next
      ck(replace_flagged(c->stream, Q.t.p, rows, n, defmask, c->seed++), "replace");
      ++c->launches;
    }
    check_finite(c, Q.t, pass == 0 ? "cholqr pass 1" : "cholqr pass >1");
  }
  dfree(c, defmask);
  return Q;
}

// FP64 truncated SVD for large matrices: randomized subspace iteration (Halko,
// Martinsson & Tropp, SIAM Rev. 53, 217 (2011)) with oversampling
// l = k + max(16, k/2), every iterate orthonormalised by the fused CholeskyQR,
// and a Rayleigh-Ritz step after each sweep: with Z = M^T Q = Qz R (CholeskyQR
// of Z, R = Qz^T Z), Q^T M = R^T Qz^T, so the left singular vectors of Q^T M
// are the right singular vectors V of the l x l matrix R (one-sided Jacobi) and
// the Ritz vectors are U = Q V.  The sweeps stop when the span of the leading k
// Ritz vectors no longer moves (RMS principal-angle sine < kSubspaceTol, or
// stagnation at the rounding floor) or after kMaxPowerIters; inside a stream
// capture the host cannot look, so kCapturedPowerIters sweeps run.
Tmp left_svd_subspace(ctm_ctx* c, const double* M, int rows, int cols, int k, int slot) {
  const int l = std::min(k + std::max(kMinOversample, k / 2), std::min(rows, cols));
  // Y = M X with X row-major cols x l: Y row-major rows x l
  auto times_M = [&](const double* X) {
    Tmp Y(c, {rows, l});
    gemm64(c, rows, l, cols, 1.0, M, lm1(rows, cols), lm1(cols, 1), X, lm1(cols, l), lm1(l, 1),
           0.0, Y.t.p, lm1(rows, l), lm1(l, 1));
    return Y;
  };
  // Z = M^T Q with Q row-major rows x l: Z row-major cols x l
  auto times_Mt = [&](const double* Qr) {
    Tmp Z(c, {cols, l});
    gemm64(c, cols, l, rows, 1.0, M, lm1(cols, 1), lm1(rows, cols), Qr, lm1(rows, l), lm1(l, 1),
           0.0, Z.t.p, lm1(cols, l), lm1(l, 1));
    return Z;
  };
  Tmp Q;
  {
    Tmp Om(c, {cols, l});
    ck(gaussian_fill(c->stream, Om.t.p, (long long)cols * l, c->seed++), "gaussian");
    ++c->launches;
    Tmp Y = times_M(Om.t.p);
    // warm start: the leading k columns start from the converged basis of the
    // previous call at this position (the oversampling columns stay random)
    if (slot >= 0) {
      const auto& ce = c->cache[slot];
      if (ce.p && ce.rows == rows && ce.k == k)
        ck(cudaMemcpy2DAsync(Y.t.p, sizeof(double) * l, ce.p, sizeof(double) * k,
                             sizeof(double) * k, rows, cudaMemcpyDeviceToDevice, c->stream),
           "warm start");
    }
    Q = cholqr(c, Y.t.p, l, 1, rows, l, 3);
  }
  const int max_iters = c->capturing ? kCapturedPowerIters : kMaxPowerIters;
  // The Rayleigh-Ritz step (an l x l Jacobi) runs on sweep 0, sweep 1 and then
  // only where the geometric rate of the subspace movement measured so far says
  // the span should have converged; the cheap part of a sweep (two products and
  // two CholeskyQRs) runs every time.
  double prev_moved = INFINITY;
  int prev_check = -1, next_check = 0;
  Tmp Uk;
  for (int it = 0; it < max_iters; ++it) {
    Tmp Z = times_Mt(Q.t.p);
    Tmp Qz = cholqr(c, Z.t.p, l, 1, cols, l, 3);
    const bool last = it + 1 == max_iters;
    if (it == next_check || last) {
      // R = Qz^T Z (l x l), stored column-major for Jacobi on its columns
      Tmp Rc(c, {l, l});
      gemm64(c, l, l, cols, 1.0, Qz.t.p, lm1(l, 1), lm1(cols, l), Z.t.p, lm1(cols, l),
             lm1(l, 1), 0.0, Rc.t.p, lm1(l, 1), lm1(l, l));
      Z.release();
      Tmp V(c, {l, l});
      jacobi(c, Rc.t.p, l, l, V.t.p);
      Tmp Vk;
      {
        Tmp sig(c, {l});
        int* perm = (int*)dalloc(c, (l + 1) / 2 + 1);
        ck(column_norms_sorted(c->stream, Rc.t.p, l, l, sig.t.p, perm), "norms");
        Vk = Tmp(c, {l, k});
        ck(gather_sorted_columns(c->stream, Vk.t.p, l, k, nullptr, V.t.p, sig.t.p, perm),
           "gather");
        c->launches += 3;
        dfree(c, perm);
      }
      Tmp Un = ein64(c, "ic,cr->ir", Q.t, Vk.t);
      const bool check = !c->capturing && prev_check >= 0;
      const double moved = check ? subspace_change(c, Uk.t.p, Un.t.p, rows, k, k) : 1.0;
      Uk = std::move(Un);
      if (trace_on() && check)
        std::fprintf(stderr, "[ctm] subspace iteration %dx%d k=%d l=%d sweep %d: moved %.3e\n",
                     rows, cols, k, l, it + 1, moved);
      // converged, or down at the rounding floor (no longer shrinking)
      if (moved < kSubspaceTol || (moved < 1e-10 && moved > 0.9 * prev_moved)) break;
      if (last) break;
      next_check = it + 1;
      if (check && std::isfinite(prev_moved) && moved < prev_moved) {
        const double rate = std::pow(moved / prev_moved, 1.0 / (it - prev_check));
        if (rate < 0.9) {
          const double sweeps = std::log(kSubspaceTol / moved) / std::log(rate);
          next_check = it + std::max(1, std::min(8, (int)std::ceil(sweeps)));
        }
      }
      prev_moved = check ? moved : INFINITY;
      prev_check = it;
    }
    Tmp Y = times_M(Qz.t.p);
    Q = cholqr(c, Y.t.p, l, 1, rows, l, 3);
  }
  if (slot >= 0 && !c->capturing) {  // keep the converged basis for the next call here
    auto& ce = c->cache[slot];
    if (!ce.p || ce.rows != rows || ce.k != k) {
      ce.p = owned_alloc(c, (long long)rows * k);
      ce.rows = rows;
      ce.k = k;
    }
    ck(cudaMemcpyAsync(ce.p, Uk.t.p, sizeof(double) * rows * k, cudaMemcpyDeviceToDevice,
                       c->stream),
       "cache");
  }
  return Uk;
}

constexpr int kColdIters = 2;  // power iterations without a cached subspace
constexpr int kWarmIters = 1;  // with the subspace cached at this position

// Leading-k left singular subspace of M (row-major rows x cols) by subspace
// iteration: Q <- orth(M (M^T Q)), products on the tensor cores in the
// context's precision, orthonormalisation by FP64 CholeskyQR.  The basis of the
// previous call at the same position (`slot`) is the starting block when it
// fits, otherwise a Gaussian sketch.  Only the subspace matters for a
// projector v v^T, so the basis is returned as it comes.
Tmp left_svd_power(ctm_ctx* c, const double* M, int rows, int cols, int k, int slot) {
  auto& ce = c->cache[slot];
  Tmp Q;
  int iters = kWarmIters;
  if (ce.p && ce.rows == rows && ce.k == k) {
    Q = Tmp(c, {rows, k});
    ck(cudaMemcpyAsync(Q.t.p, ce.p, sizeof(double) * rows * k, cudaMemcpyDeviceToDevice, c->stream),
       "cache");
  } else {
    iters = kColdIters;
    Tmp Om(c, {cols, k});
    ck(gaussian_fill(c->stream, Om.t.p, (long long)cols * k, c->seed++), "gaussian");
    ++c->launches;
    Tmp Y(c, {rows, k});
    gemm_mixed(c, rows, k, cols, M, lm1(rows, cols), lm1(cols, 1), Om.t.p, lm1(cols, k),
               lm1(k, 1), Y.t.p, lm1(rows, k), lm1(k, 1));
    Q = cholqr(c, Y.t.p, k, 1, rows, k, 4);
  }
  for (int it = 0; it < iters; ++it) {
    Tmp Z(c, {cols, k});
    gemm_mixed(c, cols, k, rows, M, lm1(cols, 1), lm1(rows, cols), Q.t.p, lm1(rows, k), lm1(k, 1),
               Z.t.p, lm1(cols, k), lm1(k, 1));
    Tmp Y(c, {rows, k});
    gemm_mixed(c, rows, k, cols, M, lm1(rows, cols), lm1(cols, 1), Z.t.p, lm1(cols, k), lm1(k, 1),
               Y.t.p, lm1(rows, k), lm1(k, 1));
    Q = cholqr(c, Y.t.p, k, 1, rows, k, 3);
  }
  if (!ce.p || ce.rows != rows || ce.k != k) {
    ce.p = owned_alloc(c, (long long)rows * k);
    ce.rows = rows;
    ce.k = k;
  }
  ck(cudaMemcpyAsync(ce.p, Q.t.p, sizeof(double) * rows * k, cudaMemcpyDeviceToDevice, c->stream),
     "cache");
  return Q;
}

// Orthonormal bases of nprob same-shape row-major matrices Y[q] (rows x n) by
// `passes` CholeskyQR passes (the first shifted), in one fused cooperative
// launch: the problems share its barriers and Cholesky latency.
void cholqr_batch(ctm_ctx* c, int nprob, const double* const* Y, Tmp* Q, int rows, int n,
                  int passes) {
  if (n > kCholqrMaxN || rows < n || nprob > kCholqrMaxProb) {
    for (int q = 0; q < nprob; ++q) Q[q] = cholqr(c, Y[q], n, 1, rows, n, passes);
    return;
  }
  double* qp[kCholqrMaxProb];
  for (int q = 0; q < nprob; ++q) {
    Q[q] = Tmp(c, {rows, n});
    qp[q] = Q[q].t.p;
  }
  Tmp W(c, {(int)cholqr_work_doubles(rows, n, nprob)});
  {
    ProfScope ps(c, 4, 0.0, true);  // flops: counted by the kernel into c->cq_flops
    const int rc = cholqr_fused_batch(c->stream, nprob, Y, qp, rows, n, passes, true, W.t.p,
                                      &c->flags->error, c->floored, c->cq_flops, c->seed,
                                      &c->launches, ps.ev0(), ps.ev1());
    c->seed += passes;
    if (rc != 0) fail(CTM_ERR_CUDA, "fused CholeskyQR launch failed");
  }
  trace_cholqr(c, W.t.p, rows, n, nprob, passes);
  for (int q = 0; q < nprob; ++q) check_finite(c, Q[q].t, "cholqr");
}

// left_svd_power for nprob matrices of one shape in lockstep (slot[q] per
// problem): the tensor-core products per problem, every orthonormalisation as
// one batched CholeskyQR.  Problems without a cached basis start from a
// Gaussian sketch; the sweep count is the largest any problem needs.
void left_svd_power_batch(ctm_ctx* c, int nprob, const double* const* M, int rows, int cols,
                          int k, const int* slot, Tmp* Q) {
  bool warm[kCholqrMaxProb];
  int iters = 0;
  bool any_cold = false;
  for (int q = 0; q < nprob; ++q) {
    auto& ce = c->cache[slot[q]];
    warm[q] = ce.p && ce.rows == rows && ce.k == k;
    iters = std::max(iters, warm[q] ? kWarmIters : kColdIters);
    any_cold = any_cold || !warm[q];
  }
  if (any_cold) {
    Tmp Y[kCholqrMaxProb];
    const double* yp[kCholqrMaxProb];
    for (int q = 0; q < nprob; ++q) {
      Y[q] = Tmp(c, {rows, k});
      if (warm[q]) {
        ck(cudaMemcpyAsync(Y[q].t.p, c->cache[slot[q]].p, sizeof(double) * rows * k,
                           cudaMemcpyDeviceToDevice, c->stream),
           "cache");
      } else {
        Tmp Om(c, {cols, k});
        ck(gaussian_fill(c->stream, Om.t.p, (long long)cols * k, c->seed++), "gaussian");
        ++c->launches;
        gemm_mixed(c, rows, k, cols, M[q], lm1(rows, cols), lm1(cols, 1), Om.t.p, lm1(cols, k),
                   lm1(k, 1), Y[q].t.p, lm1(rows, k), lm1(k, 1));
      }
      yp[q] = Y[q].t.p;
    }
    cholqr_batch(c, nprob, yp, Q, rows, k, 4);
  } else {
    for (int q = 0; q < nprob; ++q) {
      Q[q] = Tmp(c, {rows, k});
      ck(cudaMemcpyAsync(Q[q].t.p, c->cache[slot[q]].p, sizeof(double) * rows * k,
                         cudaMemcpyDeviceToDevice, c->stream),
         "cache");
    }
  }
  for (int it = 0; it < iters; ++it) {
    Tmp Y[kCholqrMaxProb];
    const double* yp[kCholqrMaxProb];
    for (int q = 0; q < nprob; ++q) {
      Tmp Z(c, {cols, k});
      gemm_mixed(c, cols, k, rows, M[q], lm1(cols, 1), lm1(rows, cols), Q[q].t.p, lm1(rows, k),
                 lm1(k, 1), Z.t.p, lm1(cols, k), lm1(k, 1));
      Y[q] = Tmp(c, {rows, k});
      gemm_mixed(c, rows, k, cols, M[q], lm1(rows, cols), lm1(cols, 1), Z.t.p, lm1(cols, k),
                 lm1(k, 1), Y[q].t.p, lm1(rows, k), lm1(k, 1));
      yp[q] = Y[q].t.p;
    }
    cholqr_batch(c, nprob, yp, Q, rows, k, 3);
  }
  for (int q = 0; q < nprob; ++q) {
    auto& ce = c->cache[slot[q]];
    if (!ce.p || ce.rows != rows || ce.k != k) {
      ce.p = owned_alloc(c, (long long)rows * k);
      ce.rows = rows;
      ce.k = k;
    }
    ck(cudaMemcpyAsync(ce.p, Q[q].t.p, sizeof(double) * rows * k, cudaMemcpyDeviceToDevice,
                       c->stream),
       "cache");
  }
}

// ---------------------------------------------------------------------------
// Environment access
// ---------------------------------------------------------------------------
inline int slot_of(int k, int r) { return (k - 1 + r) % 4; }  // stored k-1 index
inline int other(int x) { return 1 - x; }

Ten& E(ctm_ctx* c, int kind, int k, int x, int r) { return c->env[kind][slot_of(k, r)][x]; }

Ten edge_fused(const Ten& t) { return view(t, {t.dims[0], t.dims[1] * t.dims[2], t.dims[3]}); }

// Write `src` as the new (kind, k, x) of frame r into its spare buffer, normalised.
void commit(ctm_ctx* c, int kind, int k, int x, int r, const Ten& src) {
  const int s = slot_of(k, r);
  const int nb = 1 - c->cur[kind][s][x];
  double* dst = c->buf[kind][s][x][nb];
  const long long n = src.size();
  ck(cudaMemcpyAsync(dst, src.p, sizeof(double) * n, cudaMemcpyDeviceToDevice, c->stream), "commit");
  ck(normalize_f64(c->stream, dst, n, c->norm_scratch, &c->flags->bad), "normalize");
  c->launches += 2;
  Ten t;
  t.p = dst;
  t.nd = src.nd;
  for (int i = 0; i < src.nd; ++i) t.dims[i] = src.dims[i];
  c->cur[kind][s][x] = nb;
  c->env[kind][s][x] = t;
}

// ---------------------------------------------------------------------------
// Moves
// ---------------------------------------------------------------------------
// Independent factorisations run on side streams in the mixed-precision path
// (their FP64 Cholesky chains are latency-bound, so overlapping them pays).
// The host issues the branches one after the other, switching c->stream; in a
// stream capture the event edges become graph dependencies.
// Only when every factorisation of the move takes the fast path (no Jacobi,
// whose device flags a context shares between its launches).
bool can_fork(ctm_ctx* c) {
  return c->precision != CTM_FP64 && c->side[0] != nullptr && !c->prof_serial &&
         c->chi * c->D > kFastMinSide && c->chip * c->D > kFastMinSide;
}

cudaEvent_t fork_event(ctm_ctx* c) {
  if (c->fork_next == c->fork_events.size()) {
    cudaEvent_t e;
    ck(cudaEventCreateWithFlags(&e, cudaEventDisableTiming), "event");
    c->fork_events.push_back(e);
  }
  return c->fork_events[c->fork_next++];
}

// Make `to` wait for the work issued so far on `from`.
void stream_dep(ctm_ctx* c, cudaStream_t from, cudaStream_t to) {
  cudaEvent_t e = fork_event(c);
  ck(cudaEventRecord(e, from), "record");
  ck(cudaStreamWaitEvent(to, e, 0), "wait");
}

struct Proj {  // 4-index (standard) or split (sequential) isometry of one bond
  Tmp v;       // standard: [chi, D, D, k]
  Tmp v1, v2;  // sequential: [chi, D, c], [c, D, k]
};

const Ten& site(ctm_ctx* c, int r, int x, Ten& tmp) {
  tmp.p = c->site[r][x];
  tmp.nd = 5;
  tmp.dims[0] = c->d;
  for (int i = 1; i < 5; ++i) tmp.dims[i] = c->D;
  return tmp;
}

const Ten dbl_layer(ctm_ctx* c, int r, int x) {
  const int D2 = c->D * c->D;
  if (!c->dbl[r][x]) {
    Ten s;
    site(c, r, x, s);
    Tmp a = ein64(c, "puldr,pULDR->uUlLdDrR", s, s);
    double* p = owned_alloc(c, a.t.size());
    ck(cudaMemcpyAsync(p, a.t.p, sizeof(double) * a.t.size(), cudaMemcpyDeviceToDevice, c->stream),
       "dbl");
    c->dbl[r][x] = p;
  }
  Ten t;
  t.p = c->dbl[r][x];
  t.nd = 4;
  for (int i = 0; i < 4; ++i) t.dims[i] = D2;
  return t;
}

// Standard projector of the bond below x (Fig. 2c): v = leading left singular
// vectors of the upper half Q = E_L E_R of the 2x2 cell with x at top-left.
Proj projector_standard(ctm_ctx* c, int r, int x) {
  const int y = other(x), D = c->D;
  Ten ax = dbl_layer(c, r, x), ay = dbl_layer(c, r, y);
  Ten C1 = E(c, 0, 1, x, r), T1 = edge_fused(E(c, 1, 1, x, r));
  Ten T2x = edge_fused(E(c, 1, 2, x, r)), T2y = edge_fused(E(c, 1, 2, y, r));
  Ten C2 = E(c, 0, 2, y, r), T3 = edge_fused(E(c, 1, 3, y, r));
  Tmp EL;
  {
    Tmp y1 = ein(c, "dg,gUe->dUe", C1, T2x);
    Tmp y2 = ein(c, "dUe,aLd->aLUe", y1, T1);
    y1.release();
    EL = ein(c, "aLUe,ULXR->aXeR", y2, ax);
  }
  Tmp ER;
  {
    Tmp z1 = ein(c, "eUz,zh->eUh", T2y, C2);
    Tmp z2 = ein(c, "eUh,hRb->eURb", z1, T3);
    z1.release();
    ER = ein(c, "eURb,ULYR->eLbY", z2, ay);
  }
  Tmp Q = ein(c, "aXeR,eRbY->aXYb", EL, ER);
  EL.release();
  ER.release();
  const int na = Q.t.dims[0], nb = Q.t.dims[3];
  const int rows = na * D * D, cols = D * D * nb;
  const int k = std::min(c->chi, rows);
  Proj P;
  const bool fast = c->precision != CTM_FP64 && std::min(rows, cols) > kFastMinSide && k < rows &&
                    k <= cols;
  // mixed precision: subspace iteration (cache slots 48.. for the standard projectors)
  Tmp U = fast ? left_svd_power(c, Q.t.p, rows, cols, k, 48 + r * 2 + x)
               : left_svd(c, Q.t.p, rows, cols, k, 48 + r * 2 + x);
  P.v = std::move(U);
  P.v.t = view(P.v.t, {na, D, D, k});
  return P;
}

// Reduced-environment projector of the bond below x (Sec. III, Fig. 3a-b): the
// right half of the standard network is replaced by the right-move tensors
// {C2_x, T3_x} (their isometry drops out), so Q = E_L (C2_x T3_x) is a
// (chi D^2) x chi matrix.
Proj projector_reduced_env(ctm_ctx* c, int r, int x) {
  const int D = c->D;
  Ten ax = dbl_layer(c, r, x);
  Ten C1 = E(c, 0, 1, x, r), T1 = edge_fused(E(c, 1, 1, x, r));
  Ten T2x = edge_fused(E(c, 1, 2, x, r));
  Ten C2 = E(c, 0, 2, x, r), T3 = edge_fused(E(c, 1, 3, x, r));
  Tmp EL;
  {
    Tmp y1 = ein(c, "dg,gUe->dUe", C1, T2x);
    Tmp y2 = ein(c, "dUe,aLd->aLUe", y1, T1);
    y1.release();
    EL = ein(c, "aLUe,ULXR->aXeR", y2, ax);
  }
  Tmp R = ein(c, "ez,zRb->eRb", C2, T3);
  Tmp Q = ein(c, "aXeR,eRb->aXb", EL, R);
  EL.release();
  const int na = Q.t.dims[0], nb = Q.t.dims[2];
  const int rows = na * D * D, cols = nb;
  const int k = std::min(c->chi, rows);
  const bool fast = c->precision != CTM_FP64 && std::min(rows, cols) > kFastMinSide && k < rows &&
                    k <= cols;
  Proj P;
  Tmp U = fast ? left_svd_power(c, Q.t.p, rows, cols, k, 56 + r * 2 + x)
               : left_svd(c, Q.t.p, rows, cols, k, 56 + r * 2 + x);
  P.v = std::move(U);
  P.v.t = view(P.v.t, {na, D, D, k});
  return P;
}

// Split isometries from a 4-leg network Mt[alpha, k, b, beta] (Sec. IV, Fig. 4a).
// Also returns N = v1^T Mt (for reuse by the caller).
void split_projector(ctm_ctx* c, const Ten& Mt, Tmp& v1, Tmp& v2, Tmp& N, int slot) {
  const int na = Mt.dims[0], D = Mt.dims[1], nb = Mt.dims[3];
  const int k1 = std::min(c->chip, na * D);
  const bool fast = c->precision != CTM_FP64 && std::min(na * D, D * nb) > kFastMinSide;
  if (fast && k1 < na * D && k1 <= D * nb)
    v1 = left_svd_power(c, Mt.p, na * D, D * nb, k1, slot);
  else
    v1 = left_svd(c, Mt.p, na * D, D * nb, k1, slot);
  v1.t = view(v1.t, {na, D, k1});
  N = ein(c, "akc,akbz->cbz", v1, Mt);
  const int k2 = std::min(c->chi, k1 * D);
  if (fast && k2 == nb && k2 < k1 * D)  // keeps the whole column space: any orthonormal basis
    v2 = cholqr(c, N.t.p, nb, 1, k1 * D, nb, 3);
  else
    v2 = left_svd(c, N.t.p, k1 * D, nb, k2);
  v2.t = view(v2.t, {k1, D, k2});
}

// split_projector for nprob networks of one shape at once (mixed precision):
// the subspace iterations in lockstep, each orthonormalisation batched.
void split_projector_batch(ctm_ctx* c, int nprob, const Ten* Mt, Tmp* v1, Tmp* v2, Tmp* N,
                           const int* slot) {
  const int na = Mt[0].dims[0], D = Mt[0].dims[1], nb = Mt[0].dims[3];
  bool same = true;
  for (int q = 1; q < nprob; ++q)
    for (int i = 0; i < 4; ++i) same = same && Mt[q].dims[i] == Mt[0].dims[i];
  const int k1 = std::min(c->chip, na * D);
  if (!same || c->precision == CTM_FP64 || !(k1 < na * D && k1 <= D * nb)) {
    for (int q = 0; q < nprob; ++q) split_projector(c, Mt[q], v1[q], v2[q], N[q], slot[q]);
    return;
  }
  const double* mp[kCholqrMaxProb];
  for (int q = 0; q < nprob; ++q) mp[q] = Mt[q].p;
  left_svd_power_batch(c, nprob, mp, na * D, D * nb, k1, slot, v1);
  for (int q = 0; q < nprob; ++q) {
    v1[q].t = view(v1[q].t, {na, D, k1});
    N[q] = ein(c, "akc,akbz->cbz", v1[q], Mt[q]);
  }
  const int k2 = std::min(c->chi, k1 * D);
  if (k2 == nb && k2 < k1 * D) {  // the whole column space: any orthonormal basis
    const double* np[kCholqrMaxProb];
    for (int q = 0; q < nprob; ++q) np[q] = N[q].t.p;
    cholqr_batch(c, nprob, np, v2, k1 * D, nb, 3);
  } else {
    for (int q = 0; q < nprob; ++q) v2[q] = left_svd(c, N[q].t.p, k1 * D, nb, k2);
  }
  for (int q = 0; q < nprob; ++q) v2[q].t = view(v2[q].t, {k1, D, k2});
}

// Sequential ket-then-bra absorption of an edge T[prev, k, b, next] with the
// site's legs (u, l, d, r) playing the roles in `roles` ('i' in, 'o' out,
// 'p' prev, 'n' next) (Sec. IV, Fig. 4b).  Returns [chi_p, out_k, out_b, chi_n].
Tmp absorb_edge_seq(ctm_ctx* c, const Ten& T, const Ten& S, const char* roles, const Ten& vp1,
                    const Ten& vp2, const Ten& vn1, const Ten& vn2) {
  char ket[6] = {'s', 0, 0, 0, 0, 0}, bra[6] = {'s', 0, 0, 0, 0, 0};
  for (int i = 0; i < 4; ++i) {
    switch (roles[i]) {
      case 'i': ket[i + 1] = 'k'; bra[i + 1] = 'b'; break;
      case 'o': ket[i + 1] = 'o'; bra[i + 1] = 'O'; break;
      case 'p': ket[i + 1] = 'q'; bra[i + 1] = 'Q'; break;
      case 'n': ket[i + 1] = 'n'; bra[i + 1] = 'N'; break;
      default: fail(CTM_ERR_ARG, "internal: bad role");
    }
  }
  char spec[64];
  Tmp X1 = ein(c, "AkbB,Bnc->Akbnc", T, vn1);
  std::snprintf(spec, sizeof spec, "Akbnc,%s->Abcsoq", ket);
  Tmp X2 = ein(c, spec, X1, S);
  X1.release();
  Tmp X3 = ein(c, "Abcsoq,Aqe->bcsoe", X2, vp1);
  X2.release();
  Tmp X4 = ein(c, "bcsoe,cNy->bsoeNy", X3, vn2);
  X3.release();
  std::snprintf(spec, sizeof spec, "bsoeNy,%s->oeyOQ", bra);
  Tmp X5 = ein(c, spec, X4, S);
  X4.release();
  return ein(c, "oeyOQ,eQx->xoOy", X5, vp2);
}

// Reduced-network projector of the bond below x (Sec. III-IV, Fig. 3c, Fig. 8).
Proj projector_seq(ctm_ctx* c, int r, int x, int col) {
  const int base = ((r * 2 + col) * 2 + x) * 3;
  Ten S;
  site(c, r, x, S);
  Ten C1 = E(c, 0, 1, x, r), T1 = E(c, 1, 1, x, r);
  Ten C2 = E(c, 0, 2, x, r), T3 = E(c, 1, 3, x, r);
  Ten T2 = E(c, 1, 2, x, r);
  Tmp vl1, vl2, Nl, vr1, vr2, Nr;
  const cudaStream_t main = c->stream;
  const bool fork = can_fork(c);
  // P_a: L on the caller's stream, R on side 0; P_b (on side 1): R on side 2
  cudaStream_t sideR = fork ? c->side[x == 0 ? 0 : 2] : main;
  if (fork) stream_dep(c, main, sideR);
  {
    Tmp L = ein(c, "dg,akbd->gkba", C1, T1);
    split_projector(c, L, vl1, vl2, Nl, base + 0);
  }
  c->stream = sideR;
  {
    Tmp R = ein(c, "ez,zkbw->ekbw", C2, T3);
    split_projector(c, R, vr1, vr2, Nr, base + 1);
  }
  c->stream = main;
  if (fork) stream_dep(c, sideR, main);
  Tmp C1p = ein(c, "cby,cba->ya", vl2, Nl);
  Tmp C2p = ein(c, "cby,cbw->yw", vr2, Nr);
  Nl.release();
  Nr.release();
  // T'2: the top edge with x absorbed, left bond by v_l, right bond by v_r
  Tmp T2p = absorb_edge_seq(c, T2, S, "ipon", vl1, vl2, vr1, vr2);
  Tmp Xm = ein(c, "ya,ykbz->akbz", C1p, T2p);
  T2p.release();
  Tmp M = ein(c, "akbz,zw->akbw", Xm, C2p);
  Xm.release();
  Proj P;
  Tmp N;
  split_projector(c, M, P.v1, P.v2, N, base + 2);
  return P;
}

// Both reduced-network projectors of a column (Sec. III-IV, Fig. 3c, Fig. 8) in
// the mixed-precision path: the four boundary factorisations (v_l, v_r of both
// sublattices) share their orthonormalisations, then the two reduced networks do.
void projectors_seq_batched(ctm_ctx* c, int r, int col, Proj* P) {
  Ten S[2];
  Tmp L[2], R[2];
  int base[2];
  for (int x = 0; x < 2; ++x) {
    site(c, r, x, S[x]);
    base[x] = ((r * 2 + col) * 2 + x) * 3;
    L[x] = ein(c, "dg,akbd->gkba", E(c, 0, 1, x, r), E(c, 1, 1, x, r));
    R[x] = ein(c, "ez,zkbw->ekbw", E(c, 0, 2, x, r), E(c, 1, 3, x, r));
  }
  Tmp Mx[2];
  {
    const Ten mats[4] = {L[0].t, R[0].t, L[1].t, R[1].t};
    const int slots[4] = {base[0] + 0, base[0] + 1, base[1] + 0, base[1] + 1};
    Tmp v1[4], v2[4], N[4];
    split_projector_batch(c, 4, mats, v1, v2, N, slots);
    for (int x = 0; x < 2; ++x) {
      L[x].release();
      R[x].release();
    }
    for (int x = 0; x < 2; ++x) {
      const int l = 2 * x, rr = 2 * x + 1;
      Tmp C1p = ein(c, "cby,cba->ya", v2[l], N[l]);
      Tmp C2p = ein(c, "cby,cbw->yw", v2[rr], N[rr]);
      Tmp T2p = absorb_edge_seq(c, E(c, 1, 2, x, r), S[x], "ipon", v1[l], v2[l], v1[rr], v2[rr]);
      Tmp Xm = ein(c, "ya,ykbz->akbz", C1p, T2p);
      T2p.release();
      Mx[x] = ein(c, "akbz,zw->akbw", Xm, C2p);
    }
  }
  const Ten mm[2] = {Mx[0].t, Mx[1].t};
  const int slots[2] = {base[0] + 2, base[1] + 2};
  Tmp v1[2], v2[2], N[2];
  split_projector_batch(c, 2, mm, v1, v2, N, slots);
  for (int x = 0; x < 2; ++x) {
    P[x].v1 = std::move(v1[x]);
    P[x].v2 = std::move(v2[x]);
  }
}

// One column absorption in frame r (Sec. II, Fig. 2a-b).
void column_absorb(ctm_ctx* c, int r, int mode, int col) {
  Proj P[2];
  const cudaStream_t main = c->stream;
  const bool batched = mode == CTM_REDUCED_SEQUENTIAL && c->precision != CTM_FP64;
  const bool fork = !batched && mode == CTM_REDUCED_SEQUENTIAL && can_fork(c);
  if (batched) {
    projectors_seq_batched(c, r, col, P);
  } else if (fork) {
    // the two projectors are independent: P_b on side stream 1
    stream_dep(c, main, c->side[1]);
    P[0] = projector_seq(c, r, 0, col);
    c->stream = c->side[1];
    P[1] = projector_seq(c, r, 1, col);
    c->stream = main;
    stream_dep(c, c->side[1], main);
  } else {
    for (int x = 0; x < 2; ++x)
      P[x] = mode == CTM_STANDARD      ? projector_standard(c, r, x)
             : mode == CTM_REDUCED_ENV ? projector_reduced_env(c, r, x)
                                       : projector_seq(c, r, x, col);
  }
  Tmp newT[2], newC1[2], newC4[2];
  for (int x = 0; x < 2; ++x) {
    const int y = other(x);
    Ten C1 = E(c, 0, 1, x, r), T2 = E(c, 1, 2, x, r), T1 = E(c, 1, 1, x, r);
    Ten C4 = E(c, 0, 4, x, r), T4 = E(c, 1, 4, x, r);
    Ten S;
    site(c, r, x, S);
    Tmp Xc = ein(c, "dg,gkbe->dkbe", C1, T2);
    Tmp Xc4 = ein(c, "lu,rkbl->rukb", C4, T4);
    if (mode == CTM_STANDARD || mode == CTM_REDUCED_ENV) {  // double-layer absorption
      const Proj& vb = P[x];
      const Proj& vt = P[y];
      const int D2 = c->D * c->D;
      Ten ax = dbl_layer(c, r, x);
      Ten vtf = view(vt.v.t, {vt.v.t.dims[0], D2, vt.v.t.dims[3]});
      Ten vbf = view(vb.v.t, {vb.v.t.dims[0], D2, vb.v.t.dims[3]});
      Tmp W1 = ein(c, "aLu,uUn->aLUn", edge_fused(T1), vtf);
      Tmp W2 = ein(c, "aLUn,ULXR->anXR", W1, ax);
      W1.release();
      Tmp Tn = ein(c, "anXR,aXp->pRn", W2, vbf);
      newT[y] = std::move(Tn);
      newT[y].t = view(newT[y].t, {newT[y].t.dims[0], c->D, c->D, newT[y].t.dims[2]});
      newC1[y] = ein(c, "dkbe,dkby->ye", Xc, vt.v);
      newC4[y] = ein(c, "rukb,ukby->ry", Xc4, vb.v);
    } else {
      const Proj& vb = P[x];
      const Proj& vt = P[y];
      newT[y] = absorb_edge_seq(c, T1, S, "nipo", vb.v1, vb.v2, vt.v1, vt.v2);
      Tmp X2 = ein(c, "dkc,dkbe->cbe", vt.v1, Xc);
      newC1[y] = ein(c, "cby,cbe->ye", vt.v2, X2);
      Tmp W = ein(c, "rukb,ukc->rcb", Xc4, vb.v1);
      newC4[y] = ein(c, "rcb,cby->ry", W, vb.v2);
    }
  }
  for (int y = 0; y < 2; ++y) {
    commit(c, 1, 1, y, r, newT[y]);
    commit(c, 0, 1, y, r, newC1[y]);
    commit(c, 0, 4, y, r, newC4[y]);
  }
}

void check_flags(ctm_ctx* c) {
  DevFlags h;
  ck(cudaMemcpyAsync(&h, c->flags, sizeof(DevFlags), cudaMemcpyDeviceToHost, c->stream), "flags");
  ck(cudaStreamSynchronize(c->stream), "sync");
  if (h.error || h.noconv || h.bad || h.tc_timeout) {
    ck(cudaMemsetAsync(c->flags, 0, sizeof(DevFlags), c->stream), "flags reset");
    if (h.error) fail(CTM_ERR_CUDA, "a grid barrier timed out");
    if (h.tc_timeout) fail(CTM_ERR_CUDA, "a tensor-core pipeline wait timed out");
    if (h.bad) fail(CTM_ERR_NAN, "a new environment tensor was zero or not finite");
    fail(CTM_ERR_NOCONV, "a Jacobi SVD reached its sweep cap");
  }
}

bool all_bonds_at(ctm_ctx* c, int target);

// After a replay of the graph of direction dir: add its tensor-core event pairs
// to the per-class timing when that class is being timed.
void graph_account(ctm_ctx* c, int dir) {
  if (!c->prof_mask) return;
  ck(cudaStreamSynchronize(c->stream), "sync");
  for (const auto& g : c->gev[dir]) {
    if (!((c->prof_mask >> g.cls) & 1)) continue;
    float ms = 0.f;
    if (cudaEventElapsedTime(&ms, g.e0, g.e1) == cudaSuccess) c->prof[g.cls].ms += ms;
    c->prof[g.cls].count += 1;
    c->prof[g.cls].flops += g.flops;
  }
  cudaGetLastError();
}

void drop_graphs(ctm_ctx* c) {
  for (int d = 0; d < 4; ++d) {
    if (c->gexec[d]) cudaGraphExecDestroy(c->gexec[d]);
    c->gexec[d] = nullptr;
    for (auto& g : c->gev[d]) {
      cudaEventDestroy(g.e0);
      cudaEventDestroy(g.e1);
    }
    c->gev[d].clear();
    c->warm[d] = false;
  }
}

bool graph_eligible(ctm_ctx* c, int mode) {
  static int off = -1;
  if (off < 0) {
    const char* e = std::getenv("CTM_NO_GRAPHS");
    off = (e && *e && *e != '0') ? 1 : 0;
  }
  return !off && c->graphs_ok && c->stream != nullptr && c->precision != CTM_FP64 &&
         !c->prof_serial && mode == CTM_REDUCED_SEQUENTIAL && !trace_on() && !check_on() &&
         all_bonds_at(c, c->chi);
}

// Eager issue of one move (no host synchronisation).
void issue_move(ctm_ctx* c, int dir, int mode) {
  c->fork_next = 0;
  column_absorb(c, dir, mode, 0);
  column_absorb(c, dir, mode, 1);
}

// A steady-state move is a fixed launch sequence: once a direction has run
// eagerly with warm caches, its two column absorptions are captured into a
// CUDA graph and replayed (every updated tensor flips its ping-pong buffer
// twice per move, so the buffers a graph reads and writes stay the same).
void do_move(ctm_ctx* c, int dir, int mode) {
  c->fork_next = 0;
  if (graph_eligible(c, mode)) {
    if (!c->gexec[dir] && c->warm[dir]) {
      cudaGraph_t graph = nullptr;
      bool ok = cudaStreamBeginCapture(c->stream, cudaStreamCaptureModeThreadLocal) == cudaSuccess;
      if (ok) {
        c->capturing = true;
        c->capture_dir = dir;
        std::string why;
        const long long l0 = c->launches;
        try {
          column_absorb(c, dir, mode, 0);
          column_absorb(c, dir, mode, 1);
          c->glaunches[dir] = c->launches - l0;
          c->launches = l0;  // counted when the graph runs
        } catch (const CtmError& e) {
          ok = false;
          why = e.msg;
        }
        c->capturing = false;
        cudaError_t ee = cudaStreamEndCapture(c->stream, &graph);
        if (ee != cudaSuccess) {
          ok = false;
          why += std::string(" end capture: ") + cudaGetErrorString(ee);
        }
        if (ok) {
          ee = cudaGraphInstantiate(&c->gexec[dir], graph, 0);
          if (ee != cudaSuccess) {
            c->gexec[dir] = nullptr;
            ok = false;
            why += std::string(" instantiate: ") + cudaGetErrorString(ee);
          }
        }
        if (graph) cudaGraphDestroy(graph);
        if (!ok && std::getenv("CTM_GRAPH_DEBUG"))
          std::fprintf(stderr, "[ctm] graph capture of direction %d failed: %s\n", dir,
                       why.c_str());
      }
      cudaGetLastError();
      if (!ok) {  // capture not possible here: run eagerly from now on
        c->graphs_ok = false;
        drop_graphs(c);
      }
    }
    if (c->gexec[dir]) {
      if (std::getenv("CTM_GRAPH_DEBUG")) std::fprintf(stderr, "[ctm] replay graph %d\n", dir);
      ck(cudaGraphLaunch(c->gexec[dir], c->stream), "graph launch");
      c->launches += c->glaunches[dir];
      graph_account(c, dir);
      check_flags(c);
      return;
    }
  }
  column_absorb(c, dir, mode, 0);
  column_absorb(c, dir, mode, 1);
  check_flags(c);
  if (graph_eligible(c, mode)) c->warm[dir] = true;
}

bool all_bonds_at(ctm_ctx* c, int target) {
  for (int kind = 0; kind < 2; ++kind)
    for (int k = 0; k < 4; ++k)
      for (int x = 0; x < 2; ++x) {
        const Ten& t = c->env[kind][k][x];
        if (t.dims[0] < target || t.dims[t.nd - 1] < target) return false;
      }
  return true;
}

std::vector<int> all_dims(ctm_ctx* c) {
  std::vector<int> v;
  for (int kind = 0; kind < 2; ++kind)
    for (int k = 0; k < 4; ++k)
      for (int x = 0; x < 2; ++x) {
        const Ten& t = c->env[kind][k][x];
        for (int i = 0; i < t.nd; ++i) v.push_back(t.dims[i]);
      }
  return v;
}

// ---------------------------------------------------------------------------
// Initial environment
// ---------------------------------------------------------------------------
void fold_init(ctm_ctx* c) {
  const int D = c->D, D2 = D * D;
  Ten bnd;
  bnd.p = c->bnd;
  bnd.nd = 2;
  bnd.dims[0] = bnd.dims[1] = D;
  for (int k = 1; k <= 4; ++k)
    for (int x = 0; x < 2; ++x) {
      Ten Sx, Sy;
      site(c, k - 1, x, Sx);
      site(c, k - 1, other(x), Sy);
      Tmp X1 = ein64(c, "puldr,uU->pldrU", Sx, bnd);
      Tmp X2 = ein64(c, "pldrU,lL->pdrUL", X1, bnd);
      Tmp Cc = ein64(c, "pdrUL,pULDR->dDrR", X2, Sx);
      Cc.t = view(Cc.t, {D2, D2});
      commit(c, 0, k, x, 0, Cc);
      Tmp Y1 = ein64(c, "puldr,lL->pudrL", Sy, bnd);
      Tmp Tt = ein64(c, "pudrL,pULDR->dDrRuU", Y1, Sy);
      Tt.t = view(Tt.t, {D2, D, D, D2});
      commit(c, 1, k, x, 0, Tt);
    }
}

void grow(ctm_ctx* c) {
  for (int it = 0; it < 16 && !all_bonds_at(c, c->chi); ++it) {
    std::vector<int> before = all_dims(c);
    for (int dir = 0; dir < 4; ++dir) do_move(c, dir, CTM_STANDARD);
    if (all_dims(c) == before) break;
  }
}

// ---------------------------------------------------------------------------
// Observables
// ---------------------------------------------------------------------------
std::vector<double> spectrum(ctm_ctx* c, const Ten& C) {
  // singular values of the corner via one-sided Jacobi on its columns (or rows)
  int n1 = C.dims[0], n2 = C.dims[1];
  const bool cols_side = n2 <= n1;
  const int nrows = cols_side ? n1 : n2, ncols = cols_side ? n2 : n1;
  Tmp X(c, {ncols, nrows});
  LegMap m;
  if (cols_side) {  // X col-major = C columns: X[j*n1 + i] = C[i*n2 + j]
    push(m, n2, 1);
    push(m, n1, n2);
    ck(permute_f64(c->stream, X.t.p, C.p, m), "transpose");
    ++c->launches;
  } else {
    ck(cudaMemcpyAsync(X.t.p, C.p, sizeof(double) * C.size(), cudaMemcpyDeviceToDevice, c->stream),
       "copy");
  }
  {
    ProfScope ps(c, 3, 0.0);
    if (jacobi_batched(c->stream, X.t.p, nrows, ncols, 1, 0, c->flags, kMaxSweeps, &c->launches,
                       kValuesOnlyTol, true) != 0)
      fail(CTM_ERR_CUDA, "Jacobi launch failed");
  }
  Tmp sig(c, {ncols});
  int* perm = (int*)dalloc(c, (ncols + 1) / 2 + 1);
  ck(column_norms_sorted(c->stream, X.t.p, nrows, ncols, sig.t.p, perm), "norms");
  c->launches += 2;
  std::vector<double> s(ncols);
  std::vector<int> hp(ncols);
  ck(cudaMemcpyAsync(s.data(), sig.t.p, sizeof(double) * ncols, cudaMemcpyDeviceToHost, c->stream),
     "d2h");
  ck(cudaMemcpyAsync(hp.data(), perm, sizeof(int) * ncols, cudaMemcpyDeviceToHost, c->stream), "d2h");
  dfree(c, perm);
  check_flags(c);
  std::vector<double> out(ncols);
  double ss = 0.0;
  for (int i = 0; i < ncols; ++i) {
    out[i] = s[hp[i]];
    ss += out[i] * out[i];
  }
  const double nrm = std::sqrt(ss);
  if (!(nrm > 0.0)) fail(CTM_ERR_NAN, "zero corner");
  for (double& v : out) v /= nrm;
  return out;
}

// CTM_SPECTRA_PRECONDITION=0 runs the corner Jacobi on the corners themselves.
bool spectra_precondition_on() {
  static int on = -1;
  if (on < 0) {
    const char* e = std::getenv("CTM_SPECTRA_PRECONDITION");
    on = (e && *e == '0') ? 0 : 1;
  }
  return on == 1;
}

// Spectra of all 8 corners; one batched Jacobi launch when they share a shape.
std::vector<std::vector<double>> spectra_all(ctm_ctx* c) {
  std::vector<std::vector<double>> out;
  const Ten& c0 = c->env[0][0][0];
  bool same = true;
  for (int i = 1; i < 8; ++i) {
    const Ten& t = c->env[0][i / 2][i % 2];
    same = same && t.dims[0] == c0.dims[0] && t.dims[1] == c0.dims[1];
  }
  if (!same) {
    for (int i = 0; i < 8; ++i) out.push_back(spectrum(c, c->env[0][i / 2][i % 2]));
    return out;
  }
  const int n1 = c0.dims[0], n2 = c0.dims[1];
  const bool cols_side = n2 <= n1;
  const int nrows = cols_side ? n1 : n2, ncols = cols_side ? n2 : n1;
  const long long per = (long long)n1 * n2;
  Tmp X(c, {8, ncols, nrows});
  // FP32 preconditioning: the same Jacobi run in FP32 (many times the FP64 rate)
  // yields V_i with C_i V_i nearly orthogonal; V_i orthonormalised in FP64
  // (CholeskyQR) keeps the singular values of C_i V_i those of C_i, and the FP64
  // Jacobi on C_i V_i, which decides them, starts close to its end.
  const bool pre = cols_side && n2 >= 64 && spectra_precondition_on();
  Tmp Vq[8];
  int pre_sweeps = 0;
  if (pre) {
    Tmp V64(c, {8, n2, n2});
    {
      float* X32 = (float*)dalloc(c, 4 * per + 4);       // 8 n1 n2 floats
      float* V32 = (float*)dalloc(c, 4 * (long long)n2 * n2 + 4);
      int* colver = (int*)dalloc(c, 4 * (long long)(n2 + 2));
      const double* cp[8];
      double* vp[8];
      for (int i = 0; i < 8; ++i) {
        cp[i] = c->env[0][i / 2][i % 2].p;
        vp[i] = V64.t.p + (long long)i * n2 * n2;
      }
      ProfScope ps(c, 3, 0.0);
      if (jacobi_precondition_f32(c->stream, cp, n1, n2, 8, X32, V32, vp, c->flags, 30, 1e-4,
                                  1e-8, colver, &c->launches) != 0)
        fail(CTM_ERR_CUDA, "FP32 Jacobi launch failed");
      dfree(c, X32);
      dfree(c, V32);
      dfree(c, colver);
    }
    if (trace_on() && !c->capturing) {
      DevFlags h;
      ck(cudaStreamSynchronize(c->stream), "sync");
      ck(cudaMemcpy(&h, c->flags, sizeof h, cudaMemcpyDeviceToHost), "d2h");
      pre_sweeps = h.sweeps;
    }
    for (int i0 = 0; i0 < 8; i0 += kCholqrMaxProb) {
      const int nb = std::min(kCholqrMaxProb, 8 - i0);
      const double* wp[kCholqrMaxProb];
      for (int q = 0; q < nb; ++q) wp[q] = V64.t.p + (long long)(i0 + q) * n2 * n2;
      cholqr_batch(c, nb, wp, Vq + i0, n2, n2, 3);
    }
  }
  for (int i = 0; i < 8; ++i) {
    const Ten& C = c->env[0][i / 2][i % 2];
    if (pre) {  // X_i (column-major n1 x n2) = C_i (row-major) V_i (row-major)
      gemm64(c, n1, n2, n2, 1.0, C.p, lm1(n1, n2), lm1(n2, 1), Vq[i].t.p, lm1(n2, n2),
             lm1(n2, 1), 0.0, X.t.p + i * per, lm1(n1, 1), lm1(n2, n1));
    } else if (cols_side) {
      LegMap m;
      push(m, n2, 1);
      push(m, n1, n2);
      ck(permute_f64(c->stream, X.t.p + i * per, C.p, m), "transpose");
      ++c->launches;
    } else {
      ck(cudaMemcpyAsync(X.t.p + i * per, C.p, sizeof(double) * per, cudaMemcpyDeviceToDevice,
                         c->stream),
         "copy");
    }
  }
  {
    ProfScope ps(c, 3, 0.0);
    int* colver = (int*)dalloc(c, 4 * (long long)(ncols + 2));  // 8 x (ncols + 1) ints
    if (jacobi_batched(c->stream, X.t.p, nrows, ncols, 8, per, c->flags, kMaxSweeps,
                       &c->launches, kValuesOnlyTol, true, colver) != 0)
      fail(CTM_ERR_CUDA, "Jacobi launch failed");
    dfree(c, colver);
  }
  if (trace_on() && !c->capturing) {
    DevFlags h;
    ck(cudaStreamSynchronize(c->stream), "sync");
    ck(cudaMemcpy(&h, c->flags, sizeof h, cudaMemcpyDeviceToHost), "d2h");
    std::fprintf(stderr, "[ctm] spectra 8 x %dx%d FP32 sweeps=%d FP64 sweeps=%d\n", nrows,
                 ncols, pre_sweeps, h.sweeps);
  }
  Tmp sig(c, {8, ncols});
  int* perm = (int*)dalloc(c, 4 * ncols + 1);
  for (int i = 0; i < 8; ++i) {
    ck(column_norms_sorted(c->stream, X.t.p + i * per, nrows, ncols, sig.t.p + i * ncols,
                           perm + i * ncols),
       "norms");
    c->launches += 2;
  }
  std::vector<double> hs(8 * ncols);
  std::vector<int> hp(8 * ncols);
  ck(cudaMemcpyAsync(hs.data(), sig.t.p, sizeof(double) * 8 * ncols, cudaMemcpyDeviceToHost,
                     c->stream),
     "d2h");
  ck(cudaMemcpyAsync(hp.data(), perm, sizeof(int) * 8 * ncols, cudaMemcpyDeviceToHost, c->stream),
     "d2h");
  dfree(c, perm);
  check_flags(c);
  for (int i = 0; i < 8; ++i) {
    std::vector<double> v(ncols);
    double ss = 0.0;
    for (int j = 0; j < ncols; ++j) {
      v[j] = hs[i * ncols + hp[i * ncols + j]];
      ss += v[j] * v[j];
    }
    const double nrm = std::sqrt(ss);
    if (!(nrm > 0.0)) fail(CTM_ERR_NAN, "zero corner");
    for (double& x : v) x /= nrm;
    out.push_back(std::move(v));
  }
  return out;
}

double scalar_of(ctm_ctx* c, const Ten& t) {
  double v = 0.0;
  ck(cudaMemcpyAsync(&v, t.p, sizeof(double), cudaMemcpyDeviceToHost, c->stream), "d2h");
  ck(cudaStreamSynchronize(c->stream), "sync");
  return v;
}

// Two-site density matrix of the horizontal bond (x, y) in frame r, from the
// 2 x 4 window (Sec. II, Fig. 1d): left half {C1, T2, T1, C4, T4; x} and right
// half {T2, C2, T3, C3, T4; y}, each with its physical legs open.  The site's
// ket and bra layers enter one after the other (the sequential order of Sec. IV)
// instead of as the double-layer tensor, so the largest intermediate is
// chi^2 d^2 D^4 rather than chi^2 D^6 (137 GB at D = 8, chi = 256).  The long
// chi^2 side of each contraction is its column side (grid x of the GEMM).
double expect_bond(ctm_ctx* c, int bond, const double* op_host) {
  const int r = (bond >= 2) ? 1 : 0;
  const int x = bond & 1, y = other(x);
  const int d = c->d, D = c->D, D2 = D * D;
  Ten Sx, Sy;
  site(c, r, x, Sx);
  site(c, r, y, Sy);
  Tmp left;  // [e, (R_ket R_bra), k, p, P]
  {
    Tmp s2;  // [P, X_bra, R_bra, p, X_ket, R_ket, m, e]
    {
      Tmp s1;  // [p, X_ket, R_ket, m, L_bra, U_bra, e]
      {
        Tmp e1 = ein64(c, "dg,gUe->dUe", E(c, 0, 1, x, r), edge_fused(E(c, 1, 2, x, r)));
        Tmp e2 = ein64(c, "dUe,mLd->mLUe", e1, edge_fused(E(c, 1, 1, x, r)));
        const Ten& t = e2.t;
        s1 = ein64(c, "pcagh,mabcfe->pghmbfe", Sx, view(t, {t.dims[0], D, D, D, D, t.dims[3]}));
      }
      s2 = ein64(c, "Pfbij,pghmbfe->Pijpghme", Sx, s1);
    }
    Tmp bl = ein64(c, "kXl,lm->kXm", edge_fused(E(c, 1, 4, x, r)), E(c, 0, 4, x, r));
    const Ten& b = bl.t;
    left = ein64(c, "Pijpghme,kgim->ehjkpP", s2, view(b, {b.dims[0], D, D, b.dims[2]}));
  }
  Tmp right;  // [e, (L_ket L_bra), k, q, Q]
  {
    Tmp s2;  // [Q, L_bra, Y_bra, q, L_ket, Y_ket, e, t]
    {
      Tmp s1;  // [q, L_ket, Y_ket, e, V_bra, W_bra, t]
      {
        Tmp f1 = ein64(c, "eVz,zh->eVh", edge_fused(E(c, 1, 2, y, r)), E(c, 0, 2, y, r));
        Tmp f2 = ein64(c, "eVh,hWt->eVWt", f1, edge_fused(E(c, 1, 3, y, r)));
        const Ten& t = f2.t;
        s1 = ein64(c, "qaghc,eabcft->qghebft", Sy, view(t, {t.dims[0], D, D, D, D, t.dims[3]}));
      }
      s2 = ein64(c, "Qbnmf,qghebft->Qnmqghet", Sy, s1);
    }
    Tmp br = ein64(c, "ti,iYk->tYk", E(c, 0, 3, y, r), edge_fused(E(c, 1, 4, y, r)));
    const Ten& b = br.t;
    right = ein64(c, "Qnmqghet,thmk->egnkqQ", s2, view(b, {b.dims[0], D, D, b.dims[2]}));
  }
  Tmp rho = ein64(c, "eRkpP,eRkqQ->pqPQ", view(left.t, {left.t.dims[0], D2, left.t.dims[3], d, d}),
                  view(right.t, {right.t.dims[0], D2, right.t.dims[3], d, d}));
  Ten rv = view(rho.t, {d * d, d * d});
  Tmp op(c, {d * d, d * d});
  ck(cudaMemcpyAsync(op.t.p, op_host, sizeof(double) * d * d * d * d, cudaMemcpyHostToDevice,
                     c->stream),
     "h2d");
  Tmp num = ein64(c, "ij,ji->", rv, op.t);
  Tmp I = identity(c, d * d);
  Tmp den = ein64(c, "ij,ji->", rv, I.t);
  const double n = scalar_of(c, num.t), dd = scalar_of(c, den.t);
  return n / dd;
}

// Row transfer (Sec. V, Fig. 9b): strip vector V[top, k, b, bottom] absorbing
// one column (T2 above, the site with `op` between its ket and bra physical
// legs, T4 below).
Tmp strip_absorb(ctm_ctx* c, const Ten& V, int s, const Ten& op) {
  Ten S;
  site(c, 0, s, S);
  Tmp W = ein64(c, "tkbr,tKBu->kbrKBu", V, E(c, 1, 2, s, 0));
  W = ein64(c, "kbrKBu,pKkDq->brBupDq", W, S);
  W = ein64(c, "brBupDq,Pp->brBuPDq", W, op);
  W = ein64(c, "brBuPDq,PBbEQ->ruDqEQ", W, S);
  return ein64(c, "ruDqEQ,vDEr->uqQv", W, E(c, 1, 4, s, 0));
}

double strip_close(ctm_ctx* c, const Ten& V, int s) {
  Tmp X = ein64(c, "uqQv,ue->eqQv", V, E(c, 0, 2, s, 0));
  Tmp Y = ein64(c, "eqQv,eqQg->gv", X, E(c, 1, 3, s, 0));
  Tmp z = ein64(c, "gv,gv->", Y, E(c, 0, 3, s, 0));
  return scalar_of(c, z.t);
}

Tmp scaled(ctm_ctx* c, const Ten& V, double f) {
  Tmp sc(c, {1});
  sc.t.nd = 0;
  ck(cudaMemcpyAsync(sc.t.p, &f, sizeof(double), cudaMemcpyHostToDevice, c->stream), "h2d");
  ck(cudaStreamSynchronize(c->stream), "sync");  // f lives on the host stack
  return ein64(c, "tkbr,->tkbr", V, sc.t);
}

void row_correlator(ctm_ctx* c, const double* op1_h, const double* op2_h, int xmax, double* out) {
  const int d = c->d;
  Tmp op1(c, {d, d}), op2(c, {d, d}), I = identity(c, d);
  ck(cudaMemcpyAsync(op1.t.p, op1_h, sizeof(double) * d * d, cudaMemcpyHostToDevice, c->stream),
     "h2d");
  ck(cudaMemcpyAsync(op2.t.p, op2_h, sizeof(double) * d * d, cudaMemcpyHostToDevice, c->stream),
     "h2d");
  Tmp V0 = ein64(c, "dt,akbd->tkba", E(c, 0, 1, 0, 0), E(c, 1, 1, 0, 0));
  V0 = ein64(c, "tkba,ra->tkbr", V0, E(c, 0, 4, 0, 0));
  Tmp Vid = strip_absorb(c, V0, 0, I.t);
  Tmp Vop = strip_absorb(c, V0, 0, op1.t);
  for (int x = 1; x <= xmax; ++x) {
    const int s = x % 2;  // sublattice of site x (site 0 is a)
    Tmp nid = strip_absorb(c, Vid, s, I.t);
    Tmp nop = strip_absorb(c, Vop, s, I.t);
    const double z = strip_close(c, nid, s);
    const double one0 = strip_close(c, nop, s) / z;
    double onex, two;
    {
      Tmp t1 = strip_absorb(c, Vid, s, op2.t);
      onex = strip_close(c, t1, s) / z;
      Tmp t2 = strip_absorb(c, Vop, s, op2.t);
      two = strip_close(c, t2, s) / z;
    }
    if (!std::isfinite(two) || !std::isfinite(one0) || !std::isfinite(onex))
      fail(CTM_ERR_NAN, "non-finite correlator");
    out[x - 1] = two - one0 * onex;
    Tmp nn = ein64(c, "tkbr,tkbr->", nid, nid);
    const double f = 1.0 / std::sqrt(scalar_of(c, nn.t));
    Vid = scaled(c, nid, f);
    Vop = scaled(c, nop, f);
  }
}

double log_kappa(ctm_ctx* c) {
  const int x = 0, y = 1, r = 0;
  auto C = [&](int k, int s) { return E(c, 0, k, s, r); };
  auto T = [&](int k, int s) { return edge_fused(E(c, 1, k, s, r)); };
  // Z00
  Tmp a1 = ein64(c, "ab,bc->ac", C(1, x), C(2, y));
  Tmp a2 = ein64(c, "ac,cd->ad", a1, C(3, x));
  Tmp z00 = ein64(c, "ad,da->", a2, C(4, y));
  // Z20: C1x C2y T3y T3x C3x C4y T1y T1x
  Tmp b1 = ein64(c, "ab,bc->ac", C(1, x), C(2, y));
  Tmp b2 = ein64(c, "ac,cKd->aKd", b1, T(3, y));
  Tmp b3 = ein64(c, "aKd,dLe->aKLe", b2, T(3, x));
  Tmp b4 = ein64(c, "aKLe,ef->aKLf", b3, C(3, x));
  Tmp b5 = ein64(c, "aKLf,fg->aKLg", b4, C(4, y));
  Tmp b6 = ein64(c, "aKLg,gLh->aKh", b5, T(1, y));
  Tmp z20 = ein64(c, "aKh,hKa->", b6, T(1, x));
  // Z02: C1x T2x T2y C2y C3x T4x T4y C4y
  Tmp c1 = ein64(c, "ab,bKc->aKc", C(1, x), T(2, x));
  Tmp c2 = ein64(c, "aKc,cLd->aKLd", c1, T(2, y));
  Tmp c3 = ein64(c, "aKLd,de->aKLe", c2, C(2, y));
  Tmp c4 = ein64(c, "aKLe,ef->aKLf", c3, C(3, x));
  Tmp c5 = ein64(c, "aKLf,fLg->aKg", c4, T(4, x));
  Tmp c6 = ein64(c, "aKg,gKh->ah", c5, T(4, y));
  Tmp z02 = ein64(c, "ah,ha->", c6, C(4, y));
  // Z22 as an upper and a lower row
  Ten ax = dbl_layer(c, r, x), ay = dbl_layer(c, r, y);
  Tmp e1 = ein64(c, "dg,gPc->dPc", C(1, x), T(2, x));
  Tmp e2 = ein64(c, "dPc,lWd->lWPc", e1, T(1, x));
  Tmp e3 = ein64(c, "lWPc,PWXY->lcXY", e2, ax);
  Tmp f1 = ein64(c, "cQe,eh->cQh", T(2, y), C(2, y));
  Tmp f2 = ein64(c, "cQh,hRf->cQRf", f1, T(3, y));
  Tmp f3 = ein64(c, "cQRf,QYZR->cfYZ", f2, ay);
  Tmp up = ein64(c, "lcXY,cfYZ->lXfZ", e3, f3);
  Tmp g1 = ein64(c, "jk,kVl->jVl", C(4, y), T(1, y));
  Tmp g2 = ein64(c, "jVl,iUj->iUVl", g1, T(4, y));
  Tmp g3 = ein64(c, "iUVl,XVUN->ilXN", g2, ay);
  Tmp h1 = ein64(c, "gh,hTi->gTi", C(3, x), T(4, x));
  Tmp h2 = ein64(c, "gTi,fSg->fSTi", h1, T(3, x));
  Tmp h3 = ein64(c, "fSTi,ZNTS->fiZN", h2, ax);
  Tmp low = ein64(c, "ilXN,fiZN->lXfZ", g3, h3);
  Tmp z22 = ein64(c, "lXfZ,lXfZ->", up, low);
  const double v22 = scalar_of(c, z22.t), v00 = scalar_of(c, z00.t);
  const double v20 = scalar_of(c, z20.t), v02 = scalar_of(c, z02.t);
  const double ratio = v22 * v00 / (v20 * v02);
  if (!(ratio > 0.0) || !std::isfinite(ratio)) fail(CTM_ERR_NAN, "non-positive norm ratio");
  return 0.25 * std::log(ratio);
}

template <class F>
int guarded(ctm_ctx* c, F&& f) {
  try {
    f();
    if (c) c->err.clear();
    return CTM_OK;
  } catch (const CtmError& e) {
    if (c) c->err = e.msg;
    return e.code;
  } catch (const std::exception& e) {
    if (c) c->err = e.what();
    return CTM_ERR_OOM;
  }
}

void copy_in(ctm_ctx* c, double* dst, const double* src, size_t n) {
  cudaPointerAttributes at;
  cudaMemcpyKind kind = cudaMemcpyHostToDevice;
  if (cudaPointerGetAttributes(&at, src) == cudaSuccess &&
      (at.type == cudaMemoryTypeDevice || at.type == cudaMemoryTypeManaged))
    kind = cudaMemcpyDeviceToDevice;
  cudaGetLastError();
  ck(cudaMemcpyAsync(dst, src, sizeof(double) * n, kind, c->stream), "copy in");
}

// Rotated copies rot^r(A), rot^r(B), r = 1..3 (a quarter turn each:
// rot(A)[p, a1, a2, a3, a4] = A[p, a2, a3, a4, a1]).
void rotate_sites(ctm_ctx* c) {
  const int d = c->d, D = c->D;
  LegMap m;
  const long long D4 = (long long)D * D * D * D, D3 = (long long)D * D * D;
  push(m, d, D4);
  push(m, D, 1);
  push(m, D, D3);
  push(m, D, (long long)D * D);
  push(m, D, D);
  for (int r = 1; r < 4; ++r)
    for (int x = 0; x < 2; ++x) {
      ck(permute_f64(c->stream, c->site[r][x], c->site[r - 1][x], m), "rotate");
      ++c->launches;
    }
}

#include "ctm_reverse.cuh"

}  // namespace

// ===========================================================================
// C ABI
// ===========================================================================
extern "C" {

int ctm_init_env(ctm_ctx** out, const double* A, const double* B, int d, int D, int chi,
                 int chi_prime, int precision, const double* boundary, void* stream) {
  if (!out || !A || !B || d < 1 || D < 1 || chi < 1 || chi_prime < 0) return CTM_ERR_ARG;
  const bool no_grow = (precision & CTM_INIT_NO_GROW) != 0;
  precision &= ~CTM_INIT_NO_GROW;
  if (precision != CTM_FP64 && precision != CTM_TF32 && precision != CTM_BF16) return CTM_ERR_ARG;
  if ((long long)chi * D * D * chi > (1ll << 31)) return CTM_ERR_ARG;
  *out = nullptr;
  ctm_ctx* c = new (std::nothrow) ctm_ctx;
  if (!c) return CTM_ERR_OOM;
  c->stream = (cudaStream_t)stream;
  c->d = d;
  c->D = D;
  c->chi = chi;
  c->chip = chi_prime > 0 ? chi_prime : chi;
  c->precision = precision;
  int rc = guarded(c, [&] {
    int dev = 0;
    ck(cudaGetDevice(&dev), "device");
    if (!coop_stream()) fail(CTM_ERR_CUDA, "cooperative stream");
    cudaMemPool_t pool;
    if (cudaDeviceGetDefaultMemPool(&pool, dev) == cudaSuccess) {
      unsigned long long thr = ~0ull;
      cudaMemPoolSetAttribute(pool, cudaMemPoolAttrReleaseThreshold, &thr);
    }
    cudaGetLastError();
    void* f = nullptr;
    ck(cudaMalloc(&f, sizeof(DevFlags)), "flags");
    c->owned.push_back(f);
    c->flags = (DevFlags*)f;
    ck(cudaMemsetAsync(c->flags, 0, sizeof(DevFlags), c->stream), "flags");
    c->norm_scratch = owned_alloc(c, kNormScratch);
    c->floored = (int*)owned_alloc(c, 1);  // two ints: floored pivots, scratch counter
    ck(cudaMemsetAsync(c->floored, 0, 2 * sizeof(int), c->stream), "floored");
    c->cq_flops = owned_alloc(c, 1);
    ck(cudaMemsetAsync(c->cq_flops, 0, sizeof(double), c->stream), "cq_flops");
    if (precision != CTM_FP64) {
      c->tc = tc_create();
      if (!c->tc) fail(CTM_ERR_UNSUPPORTED, "tensor-core GEMM unavailable");
      for (auto& st : c->side) ck(cudaStreamCreateWithFlags(&st, cudaStreamNonBlocking), "stream");
    }
    const long long ns = (long long)d * D * D * D * D;
    for (int r = 0; r < 4; ++r)
      for (int x = 0; x < 2; ++x) c->site[r][x] = owned_alloc(c, ns);
    copy_in(c, c->site[0][0], A, ns);
    copy_in(c, c->site[0][1], B, ns);
    rotate_sites(c);
    c->bnd = owned_alloc(c, (long long)D * D);
    if (boundary) {
      copy_in(c, c->bnd, boundary, (size_t)D * D);
    } else {
      ck(fill_identity(c->stream, c->bnd, D), "identity");
      ++c->launches;
    }
    const int cmax = std::max(chi, D * D);
    for (int kind = 0; kind < 2; ++kind)
      for (int k = 0; k < 4; ++k)
        for (int x = 0; x < 2; ++x)
          for (int b = 0; b < 2; ++b)
            c->buf[kind][k][x][b] =
                owned_alloc(c, kind == 0 ? (long long)cmax * cmax : (long long)cmax * D * D * cmax);
    fold_init(c);
    check_flags(c);
    if (!no_grow) grow(c);
  });
  if (rc != CTM_OK) {
    ctm_free(c);
    return rc;
  }
  *out = c;
  return CTM_OK;
}

int ctm_move(ctm_ctx* c, int dir, int mode) {
  if (!c || dir < 0 || dir > 3 ||
      (mode != CTM_STANDARD && mode != CTM_REDUCED_SEQUENTIAL && mode != CTM_REDUCED_ENV))
    return CTM_ERR_ARG;
  return guarded(c, [&] { do_move(c, dir, mode); });
}

int ctm_converge(ctm_ctx* c, int mode, int max_iter, double tol, int* iters_done,
                 double* last_delta) {
  if (!c || max_iter < 1 ||
      (mode != CTM_STANDARD && mode != CTM_REDUCED_SEQUENTIAL && mode != CTM_REDUCED_ENV))
    return CTM_ERR_ARG;
  bool converged = false;
  int rc = guarded(c, [&] {
    std::vector<std::vector<double>> old = spectra_all(c);
    double delta = INFINITY;
    int it = 0;
    for (it = 1; it <= max_iter; ++it) {
      for (int dir = 0; dir < 4; ++dir) do_move(c, dir, mode);
      delta = 0.0;
      std::vector<std::vector<double>> all = spectra_all(c);
      for (int i = 0; i < 8; ++i) {
        std::vector<double>& s = all[i];
        const size_t n = std::max(s.size(), old[i].size());
        double acc = 0.0;
        for (size_t j = 0; j < n; ++j) {
          const double a = j < s.size() ? s[j] : 0.0, b = j < old[i].size() ? old[i][j] : 0.0;
          acc += (a - b) * (a - b);
        }
        delta = std::max(delta, std::sqrt(acc));
        old[i] = std::move(s);
      }
      if (delta < tol) {
        converged = true;
        break;
      }
    }
    if (iters_done) *iters_done = std::min(it, max_iter);
    if (last_delta) *last_delta = delta;
  });
  if (rc == CTM_OK && !converged) {
    c->err = "max_iter reached";
    return CTM_ERR_NOCONV;
  }
  return rc;
}

int ctm_expect_bond(ctm_ctx* c, int bond, const double* op, double* value) {
  if (!c || bond < 0 || bond > 3 || !op || !value) return CTM_ERR_ARG;
  return guarded(c, [&] { *value = expect_bond(c, bond, op); });
}

int ctm_corner_spectrum(ctm_ctx* c, int corner, double* s, int* len) {
  if (!c || corner < 0 || corner > 7 || !s || !len) return CTM_ERR_ARG;
  return guarded(c, [&] {
    std::vector<double> v = spectrum(c, c->env[0][corner / 2][corner % 2]);
    for (size_t i = 0; i < v.size(); ++i) s[i] = v[i];
    *len = (int)v.size();
  });
}

int ctm_corner_spectra(ctm_ctx* c, double* s, int maxlen, int* lens) {
  if (!c || !s || !lens || maxlen < 1) return CTM_ERR_ARG;
  return guarded(c, [&] {
    std::vector<std::vector<double>> all = spectra_all(c);
    for (int i = 0; i < 8; ++i) {
      const int n = std::min((int)all[i].size(), maxlen);
      for (int j = 0; j < n; ++j) s[(long long)i * maxlen + j] = all[i][j];
      lens[i] = n;
    }
  });
}

int ctm_correlator(ctm_ctx* c, const double* op1, const double* op2, int xmax, double* out) {
  if (!c || !op1 || !op2 || !out || xmax < 1) return CTM_ERR_ARG;
  return guarded(c, [&] { row_correlator(c, op1, op2, xmax, out); });
}

int ctm_log_kappa(ctm_ctx* c, double* value) {
  if (!c || !value) return CTM_ERR_ARG;
  return guarded(c, [&] { *value = log_kappa(c); });
}

int ctm_get_tensor(ctm_ctx* c, int kind, int k, int x, double* out, int* dims) {
  if (!c || kind < 0 || kind > 1 || k < 1 || k > 4 || x < 0 || x > 1 || !dims) return CTM_ERR_ARG;
  return guarded(c, [&] {
    const Ten& t = c->env[kind][k - 1][x];
    for (int i = 0; i < 4; ++i) dims[i] = i < t.nd ? t.dims[i] : 0;
    if (out) {
      ck(cudaMemcpyAsync(out, t.p, sizeof(double) * t.size(), cudaMemcpyDeviceToHost, c->stream),
         "d2h");
      ck(cudaStreamSynchronize(c->stream), "sync");
    }
  });
}

int ctm_set_tensor(ctm_ctx* c, int kind, int k, int x, const double* in, const int* dims) {
  if (!c || kind < 0 || kind > 1 || k < 1 || k > 4 || x < 0 || x > 1 || !in || !dims)
    return CTM_ERR_ARG;
  const int nd = kind == 0 ? 2 : 4;
  const int cmax = std::max(c->chi, c->D * c->D);
  if (dims[0] < 1 || dims[0] > cmax || dims[nd - 1] < 1 || dims[nd - 1] > cmax) return CTM_ERR_ARG;
  if (nd == 4 && (dims[1] != c->D || dims[2] != c->D)) return CTM_ERR_ARG;
  return guarded(c, [&] {
    drop_graphs(c);  // recorded graphs assume the current shapes and buffers
    Ten& t = c->env[kind][k - 1][x];
    t.nd = nd;
    for (int i = 0; i < nd; ++i) t.dims[i] = dims[i];
    ck(cudaMemcpyAsync(t.p, in, sizeof(double) * t.size(), cudaMemcpyHostToDevice, c->stream),
       "h2d");
    ck(cudaStreamSynchronize(c->stream), "sync");
  });
}

int ctm_set_sites(ctm_ctx* c, const double* A, const double* B) {
  if (!c || !A || !B) return CTM_ERR_ARG;
  return guarded(c, [&] {
    drop_graphs(c);  // recorded graphs read the old site tensors
    const long long ns = (long long)c->d * c->D * c->D * c->D * c->D;
    copy_in(c, c->site[0][0], A, ns);
    copy_in(c, c->site[0][1], B, ns);
    rotate_sites(c);
    // double-layer tensors built so far are rebuilt in place
    for (int r = 0; r < 4; ++r)
      for (int x = 0; x < 2; ++x) {
        if (!c->dbl[r][x]) continue;
        Ten sx;
        site(c, r, x, sx);
        Tmp a = ein64(c, "puldr,pULDR->uUlLdDrR", sx, sx);
        ck(cudaMemcpyAsync(c->dbl[r][x], a.t.p, sizeof(double) * a.t.size(),
                           cudaMemcpyDeviceToDevice, c->stream),
           "dbl");
      }
    ck(cudaStreamSynchronize(c->stream), "sync");
  });
}

int ctm_energy_grad(ctm_ctx* c, int iters, double eps, const double* op, double* energy,
                    double* gA, double* gB) {
  if (!c || iters < 0 || !(eps >= 0.0) || !op || !energy) return CTM_ERR_ARG;
  return guarded(c, [&] {
    const long long ns = (long long)c->d * c->D * c->D * c->D * c->D;
    Tmp ga(c, {(int)ns}), gb(c, {(int)ns});
    const double E = energy_grad(c, iters, eps, op, ga, gb);
    if (gA)
      ck(cudaMemcpyAsync(gA, ga.t.p, sizeof(double) * ns, cudaMemcpyDefault, c->stream), "grad");
    if (gB)
      ck(cudaMemcpyAsync(gB, gb.t.p, sizeof(double) * ns, cudaMemcpyDefault, c->stream), "grad");
    ck(cudaStreamSynchronize(c->stream), "sync");
    check_flags(c);
    *energy = E;
  });
}

long long ctm_kernel_launches(ctm_ctx* c) { return c ? c->launches : 0; }

}  // extern "C"

struct ctm_batch {
  std::vector<ctm_ctx*> ctx;
  cudaStream_t master = nullptr;
  cudaGraphExec_t g[4][3] = {};
  long long glaunch[4][3] = {};
  bool warm[4][3] = {};
  bool ok = true;
  std::vector<cudaEvent_t> ev;
  std::string err;
};

namespace {

cudaEvent_t batch_event(ctm_batch* b, size_t i) {
  while (b->ev.size() <= i) {
    cudaEvent_t e;
    ck(cudaEventCreateWithFlags(&e, cudaEventDisableTiming), "event");
    b->ev.push_back(e);
  }
  return b->ev[i];
}

bool batch_eligible(ctm_batch* b, int mode) {
  for (ctm_ctx* c : b->ctx)
    if (!graph_eligible(c, mode) || c->prof_mask != 0) return false;
  return b->ok;
}

// Every state's move of direction dir on its own stream, as one graph forked
// from and joined to the batch's master stream (or eagerly until warm).
void batch_move(ctm_batch* b, int dir, int mode) {
  const int n = (int)b->ctx.size();
  if (batch_eligible(b, mode)) {
    if (!b->g[dir][mode] && b->warm[dir][mode]) {
      cudaGraph_t graph = nullptr;
      bool ok = cudaStreamBeginCapture(b->master, cudaStreamCaptureModeThreadLocal) == cudaSuccess;
      long long nk = 0;
      if (ok) {
        try {
          for (int i = 0; i < n; ++i) {
            ctm_ctx* c = b->ctx[i];
            cudaEvent_t e = batch_event(b, 2 * i);
            ck(cudaEventRecord(e, b->master), "record");
            ck(cudaStreamWaitEvent(c->stream, e, 0), "wait");
            const long long l0 = c->launches;
            issue_move(c, dir, mode);
            nk += c->launches - l0;
            c->launches = l0;
            cudaEvent_t j = batch_event(b, 2 * i + 1);
            ck(cudaEventRecord(j, c->stream), "record");
            ck(cudaStreamWaitEvent(b->master, j, 0), "wait");
          }
        } catch (const CtmError&) {
          ok = false;
        }
        if (cudaStreamEndCapture(b->master, &graph) != cudaSuccess) ok = false;
        if (ok && cudaGraphInstantiate(&b->g[dir][mode], graph, 0) != cudaSuccess) {
          b->g[dir][mode] = nullptr;
          ok = false;
        }
        if (graph) cudaGraphDestroy(graph);
      }
      cudaGetLastError();
      if (!ok) b->ok = false;
      b->glaunch[dir][mode] = nk;
    }
    if (b->g[dir][mode]) {
      ck(cudaGraphLaunch(b->g[dir][mode], b->master), "graph launch");
      cudaEvent_t e = batch_event(b, 2 * n);
      ck(cudaEventRecord(e, b->master), "record");
      for (ctm_ctx* c : b->ctx) ck(cudaStreamWaitEvent(c->stream, e, 0), "wait");
      b->ctx[0]->launches += b->glaunch[dir][mode];
      for (ctm_ctx* c : b->ctx) check_flags(c);
      return;
    }
  }
  for (ctm_ctx* c : b->ctx) issue_move(c, dir, mode);  // concurrent on the states' streams
  for (ctm_ctx* c : b->ctx) check_flags(c);
  if (batch_eligible(b, mode)) b->warm[dir][mode] = true;
}

}  // namespace

extern "C" {

int ctm_batch_create(ctm_batch** out, ctm_ctx** ctxs, int n) {
  if (!out || !ctxs || n < 1) return CTM_ERR_ARG;
  for (int i = 0; i < n; ++i)
    if (!ctxs[i]) return CTM_ERR_ARG;
  ctm_batch* b = new (std::nothrow) ctm_batch;
  if (!b) return CTM_ERR_OOM;
  b->ctx.assign(ctxs, ctxs + n);
  if (cudaStreamCreateWithFlags(&b->master, cudaStreamNonBlocking) != cudaSuccess) {
    cudaGetLastError();
    delete b;
    return CTM_ERR_CUDA;
  }
  *out = b;
  return CTM_OK;
}

int ctm_batch_move(ctm_batch* b, int dir, int mode) {
  if (!b || dir < 0 || dir > 3 ||
      (mode != CTM_STANDARD && mode != CTM_REDUCED_SEQUENTIAL && mode != CTM_REDUCED_ENV))
    return CTM_ERR_ARG;
  try {
    batch_move(b, dir, mode);
    b->err.clear();
    return CTM_OK;
  } catch (const CtmError& e) {
    b->err = e.msg;
    return e.code;
  } catch (const std::exception& e) {
    b->err = e.what();
    return CTM_ERR_OOM;
  }
}

const char* ctm_batch_last_error(ctm_batch* b) { return b ? b->err.c_str() : "null batch"; }

void ctm_batch_free(ctm_batch* b) {
  if (!b) return;
  if (b->master) cudaStreamSynchronize(b->master);
  for (auto& row : b->g)
    for (auto& g : row)
      if (g) cudaGraphExecDestroy(g);
  for (cudaEvent_t e : b->ev) cudaEventDestroy(e);
  if (b->master) cudaStreamDestroy(b->master);
  cudaGetLastError();
  delete b;
}

int ctm_contract_test(int precision, long long M, long long N, long long K, const double* A,
                      const double* B, double* C) {
  if (M < 1 || N < 1 || K < 1 || !A || !B || !C) return CTM_ERR_ARG;
  if (precision != CTM_FP64 && precision != CTM_TF32 && precision != CTM_BF16) return CTM_ERR_ARG;
  double *dA = nullptr, *dB = nullptr, *dC = nullptr;
  TcGemm* tc = nullptr;
  int rc = CTM_OK;
  long long launches = 0;
  auto bail = [&](int code) {
    rc = code;
    return;
  };
  do {
    if (cudaMalloc(&dA, sizeof(double) * M * K) != cudaSuccess ||
        cudaMalloc(&dB, sizeof(double) * K * N) != cudaSuccess ||
        cudaMalloc(&dC, sizeof(double) * M * N) != cudaSuccess) {
      bail(CTM_ERR_OOM);
      break;
    }
    cudaMemcpy(dA, A, sizeof(double) * M * K, cudaMemcpyHostToDevice);
    cudaMemcpy(dB, B, sizeof(double) * K * N, cudaMemcpyHostToDevice);
    cudaMemset(dC, 0, sizeof(double) * M * N);
    LegMap Am, Ak, Bk, Bn, Cm, Cn;
    Am.n = Ak.n = Bk.n = Bn.n = Cm.n = Cn.n = 1;
    Am.dim[0] = Cm.dim[0] = (int)M;
    Ak.dim[0] = Bk.dim[0] = (int)K;
    Bn.dim[0] = Cn.dim[0] = (int)N;
    Am.stride[0] = K;
    Ak.stride[0] = 1;
    Bk.stride[0] = N;
    Bn.stride[0] = 1;
    Cm.stride[0] = N;
    Cn.stride[0] = 1;
    if (precision == CTM_FP64) {
      if (gemm_f64(0, M, N, K, 1.0, dA, Am, Ak, dB, Bk, Bn, 0.0, dC, Cm, Cn) != cudaSuccess) {
        bail(CTM_ERR_CUDA);
        break;
      }
    } else {
      tc = tc_create();
      if (!tc) {
        bail(CTM_ERR_UNSUPPORTED);
        break;
      }
      if (tc_contract(tc, 0, precision, M, N, K, dA, Am, Ak, dB, Bk, Bn, dC, Cm, Cn, &launches,
                      nullptr, nullptr, nullptr) != 0) {
        bail(CTM_ERR_CUDA);
        break;
      }
      if (tc_error(tc, 0) != 0) {
        bail(CTM_ERR_CUDA);
        break;
      }
    }
    if (cudaMemcpy(C, dC, sizeof(double) * M * N, cudaMemcpyDeviceToHost) != cudaSuccess)
      bail(CTM_ERR_CUDA);
  } while (false);
  cudaDeviceSynchronize();
  if (cudaGetLastError() != cudaSuccess && rc == CTM_OK) rc = CTM_ERR_CUDA;
  cudaFree(dA);
  cudaFree(dB);
  cudaFree(dC);
  tc_destroy(tc);
  return rc;
}

int ctm_truncated_svd_test(int path, const double* M, int rows, int cols, int k, double* U) {
  if (!M || !U || rows < 1 || cols < 1 || k < 1 || k > std::min(rows, cols) || path < 0 ||
      path > 2)
    return CTM_ERR_ARG;
  ctm_ctx* c = new (std::nothrow) ctm_ctx;
  if (!c) return CTM_ERR_OOM;
  int rc = guarded(c, [&] {
    void* f = nullptr;
    ck(cudaMalloc(&f, sizeof(DevFlags)), "flags");
    c->owned.push_back(f);
    c->flags = (DevFlags*)f;
    ck(cudaMemset(c->flags, 0, sizeof(DevFlags)), "flags");
    if (!coop_stream()) fail(CTM_ERR_CUDA, "cooperative stream");
    double* dM = owned_alloc(c, (long long)rows * cols);
    ck(cudaMemcpy(dM, M, sizeof(double) * (size_t)rows * cols, cudaMemcpyHostToDevice), "h2d");
    Tmp Uk = left_svd_impl(c, dM, rows, cols, k, path);
    if (Uk.t.size() != (long long)rows * k) fail(CTM_ERR_ARG, "internal: factor shape");
    ck(cudaMemcpyAsync(U, Uk.t.p, sizeof(double) * (size_t)rows * k, cudaMemcpyDeviceToHost,
                       c->stream),
       "d2h");
    Uk.release();
    check_flags(c);
  });
  ctm_free(c);
  return rc;
}

int ctm_cholqr_test(const double* Y, int rows, int n, int passes, double* Q) {
  if (!Y || !Q || rows < 1 || n < 1 || n > rows || passes < 1 || passes > 8) return CTM_ERR_ARG;
  ctm_ctx* c = new (std::nothrow) ctm_ctx;
  if (!c) return CTM_ERR_OOM;
  int rc = guarded(c, [&] {
    void* f = nullptr;
    ck(cudaMalloc(&f, sizeof(DevFlags)), "flags");
    c->owned.push_back(f);
    c->flags = (DevFlags*)f;
    ck(cudaMemset(c->flags, 0, sizeof(DevFlags)), "flags");
    c->floored = (int*)owned_alloc(c, 1);
    ck(cudaMemset(c->floored, 0, 2 * sizeof(int)), "floored");
    if (!coop_stream()) fail(CTM_ERR_CUDA, "cooperative stream");
    double* dY = owned_alloc(c, (long long)rows * n);
    ck(cudaMemcpy(dY, Y, sizeof(double) * (size_t)rows * n, cudaMemcpyHostToDevice), "h2d");
    Tmp Qd = cholqr(c, dY, n, 1, rows, n, passes);
    ck(cudaMemcpyAsync(Q, Qd.t.p, sizeof(double) * (size_t)rows * n, cudaMemcpyDeviceToHost,
                       c->stream),
       "d2h");
    Qd.release();
    check_flags(c);
  });
  ctm_free(c);
  return rc;
}

int ctm_profile_enable(ctm_ctx* c, int on) {
  if (!c) return CTM_ERR_ARG;
  return guarded(c, [&] {
    prof_collect(c);
    for (auto& pc : c->prof) {
      pc.count = 0;
      pc.ms = pc.flops = 0.0;
    }
    ck(cudaMemcpy(&c->cq_flops_base, c->cq_flops, sizeof(double), cudaMemcpyDeviceToHost),
       "cq_flops");
    const bool serial = (on & CTM_PROFILE_SERIAL) != 0;
    if ((on & kProfMaskAll) != c->prof_mask || serial != c->prof_serial)
      drop_graphs(c);  // re-capture with the new event set
    c->prof_mask = on & kProfMaskAll;
    c->prof_serial = serial;
  });
}

int ctm_profile_read(ctm_ctx* c, int cls, long long* launches, double* ms, double* flops) {
  if (!c || cls < 0 || cls >= kProfClasses || !launches || !ms || !flops) return CTM_ERR_ARG;
  return guarded(c, [&] {
    prof_collect(c);
    *launches = c->prof[cls].count;
    *ms = c->prof[cls].ms;
    *flops = c->prof[cls].flops;
    if (cls == 4 && ((c->prof_mask >> 4) & 1)) {  // every CholeskyQR launch is timed then
      double now = 0.0;
      ck(cudaMemcpy(&now, c->cq_flops, sizeof(double), cudaMemcpyDeviceToHost), "cq_flops");
      *flops = now - c->cq_flops_base;
    }
  });
}

const char* ctm_last_error(ctm_ctx* c) { return c ? c->err.c_str() : "null context"; }

void ctm_free(ctm_ctx* c) {
  if (!c) return;
  cudaStreamSynchronize(c->stream);
  for (void* p : c->owned) cudaFree(p);
  drop_graphs(c);
  for (auto& st : c->side)
    if (st) cudaStreamDestroy(st);
  for (cudaEvent_t e : c->fork_events) cudaEventDestroy(e);
  if (c->tc) tc_destroy(c->tc);
  for (auto& pc : c->prof)
    for (cudaEvent_t e : pc.ev) cudaEventDestroy(e);
  cudaGetLastError();
  delete c;
}

}  // extern "C"
