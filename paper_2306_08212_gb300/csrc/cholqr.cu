// Fused CholeskyQR in FP64: an orthonormal basis Q (row-major rows x n) of the
// columns of Y (row-major rows x n) in ONE cooperative launch, every pass of
// the method inside it, phases separated by bounded grid barriers.
//
// One pass (scaled CholeskyQR; Fukaya, Kannan, Nakatsukasa, Yamamoto &
// Yanagisawa, SIAM J. Sci. Comput. 42, A477 (2020), for the shifted first pass):
//   G  = X^T X                          Gram, 32 x 32 tiles x row chunks, partial
//                                        tiles reduced in a fixed order (deterministic)
//   G' = D^-1 G D^-1 (+ s I)            D = diag(sqrt(G_ii)); shift s on the first
//                                        pass of an ill-conditioned input
//   G' = L L^T                          right-looking blocked Cholesky, 32-wide
//                                        panels; the diagonal block and its inverse
//                                        on one CTA per problem
//   Q  = X D^-1 L^-T                    blocked forward substitution, each CTA
//                                        owning 16-row blocks (no barrier inside)
// When G' is within kNearIdentity of the identity (max |G' - I|, decided on the
// device from the reduced Gram), L^-T = I - U + O(e^2) with U the strict upper
// triangle of G' - I: the error e^2 <= 1e-16 is below FP64 rounding, so that
// pass skips the Cholesky and computes Q = X D^-1 (I - U) directly; below
// kOrthonormal the input is orthonormal already and the pass only rescales it.
//
// Passes stop early per problem: an unshifted pass whose scaled Gram has
// ||G' - I||_F <= kLastPassFro has kappa(G') <= (1 + f) / (1 - f) <= 3, so its
// output is orthonormal to a small multiple of n u (the CholeskyQR bound is
// proportional to kappa^2) and a further pass would not change it.
//
// Rank deficiency (unshifted passes): a pivot of the scaled Gram below tau marks
// a column in the span of the earlier ones; its L column becomes e_k and, after a
// pass that is neither the first nor the last, the column is replaced by
// Gaussian values (counter-based SplitMix64 + Box-Muller) that the next pass
// orthonormalises against the rest.
//
// FP64 on GB300 retires about two FMA per clock per SM, so every phase is
// bound by FP64 issue: the Gram and the substitution each cost rows n^2 / 2 FMA,
// spread over all SMs; the Cholesky costs n^3 / 6, most of it latency.
#include <cuda_runtime.h>

#include <cmath>
#include <cstdlib>
#include <vector>

#include "ctm_internal.h"

namespace ctm {

namespace {

constexpr int kCqThreads = 256;
constexpr int kTb = 32;           // tile / panel width
constexpr int kRowBlock = 16;     // rows per substitution block (two per thread column)
constexpr double kNearIdentity = 1e-8;
constexpr double kOrthonormal = 1e-14;  // max |G' - I| of an input taken as orthonormal
constexpr double kLastPassFro = 0.5;    // ||G' - I||_F that makes a pass the last one
constexpr long long kCqBarrierLimit = 4000000000ll;  // clocks (~2 s)
constexpr int kCqMaxN = kCholqrMaxN;

constexpr int kCqMaxProb = kCholqrMaxProb;  // independent problems of one launch
constexpr int kPitch = kTb + 1;             // shared-memory row pitch of 32-wide tiles

// Every phase takes its shared memory from the one dynamic buffer (the phases
// are separated by barriers), so that two CTAs fit on an SM when n <= 256.
__device__ __forceinline__ double* cq_smem() {
  extern __shared__ double cq_dyn[];
  return cq_dyn;
}

// dynamic shared memory of a launch for n columns: the larger of the substitution
// phase (two 16-row blocks of the rows and two tiles) and the diagonal factor
// (three 32 x 32 tiles)
__host__ __device__ constexpr size_t cq_smem_doubles(int n) {
  return (size_t)2 * kRowBlock * n + kTb * kPitch + kRowBlock * kPitch > (size_t)3 * kTb * kPitch + 2 * kTb
             ? (size_t)2 * kRowBlock * n + kTb * kPitch + kRowBlock * kPitch
             : (size_t)3 * kTb * kPitch + 2 * kTb;
}

// Per-problem pointers (inputs, outputs and this problem's part of the work buffer).
struct CqProb {
  const double* Y;
  double* Q;
  double* part;     // [nchunk][npairs][32 * 32]
  double* G;        // n x n, lower triangle used
  double* Linv;     // [T][32 * 32]
  double* dscale;   // n
  double* dinv;     // n, 1 / dscale
  double* emax;     // [passes] max |G' - I| (bits of a non-negative double)
  double* fro2;     // [passes] ||G' - I||_F^2
  int* defmask;     // n
};

struct CqArgs {
  int nprob;
  int rows, n, passes, shifted;
  int nchunk, chunk_rows, npairs, T;
  CqProb prob[kCqMaxProb];
  DevFlags* fl;     // this launch's own barrier words (inside the work buffer)
  int* err_out;     // sticky error word of the caller (set on a barrier timeout)
  int* floored;
  double* flops_out;  // executed FP64 flops are added here (may be null)
  unsigned long long* stamps;  // diagnostics (may be null): [0] count, then (tag, ns) pairs
  unsigned long long seed;
};

__device__ __forceinline__ unsigned cq_ld_acquire(const unsigned* p) {
  unsigned v;
  asm volatile("ld.acquire.gpu.global.u32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
  return v;
}

__device__ __forceinline__ unsigned cq_atom_add_release(unsigned* p, unsigned v) {
  unsigned old;
  asm volatile("atom.add.release.gpu.global.u32 %0, [%1], %2;" : "=r"(old) : "l"(p), "r"(v)
               : "memory");
  return old;
}

// Generation barrier over the whole grid with a clock limit; false once any
// block has timed out (every block then returns).
__device__ bool cq_barrier(DevFlags* fl) {
  __shared__ int s_ok;
  __syncthreads();
  if (threadIdx.x == 0) {
    __threadfence();
    const unsigned g = cq_ld_acquire(&fl->bar_gen);
    const unsigned arrived = cq_atom_add_release(&fl->bar_count, 1u);
    if (arrived == gridDim.x - 1) {
      atomicExch(&fl->bar_count, 0u);
      cq_atom_add_release(&fl->bar_gen, 1u);
    } else {
      const long long t0 = clock64();
      while (cq_ld_acquire(&fl->bar_gen) == g) {
        if (clock64() - t0 > kCqBarrierLimit) {
          atomicExch(&fl->error, 1);
          break;
        }
      }
    }
    s_ok = (*(volatile int*)&fl->error) == 0;
  }
  __syncthreads();
  return s_ok;
}

__device__ __forceinline__ unsigned long long cq_splitmix64(unsigned long long z) {
  z += 0x9E3779B97F4A7C15ull;
  z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
  z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
  return z ^ (z >> 31);
}

__device__ __forceinline__ double cq_gauss(unsigned long long seed, unsigned long long idx) {
  const unsigned long long base = seed * 0xD1B54A32D192ED03ull + 2ull * idx;
  const unsigned long long z1 = cq_splitmix64(base), z2 = cq_splitmix64(base + 1ull);
  const double u1 = ((double)(z1 >> 11) + 1.0) * 0x1.0p-53;
  const double u2 = (double)(z2 >> 11) * 0x1.0p-53;
  return sqrt(-2.0 * log(u1)) * cospi(2.0 * u2);
}

// (bi, bj), bi <= bj, of upper-triangle tile pair number `pair` (row-major order).
__device__ __forceinline__ void pair_of(int pair, int T, int& bi, int& bj) {
  int i = 0, start = 0;
  while (pair >= start + (T - i)) {
    start += T - i;
    ++i;
  }
  bi = i;
  bj = i + (pair - start);
}

__device__ __forceinline__ int pair_index(int bi, int bj, int T) {  // bi <= bj
  return bi * T - bi * (bi - 1) / 2 + (bj - bi);
}

// Phase G: partial Gram tiles of every problem.  Thread (ty, tx) of a 16 x 16
// layout owns the 2 x 2 outputs (2ty + a, 2tx + b) of the 32 x 32 tile.
__device__ void gram_partials(const CqArgs& a, int pass, const int* act, int nact) {
  double* As = cq_smem();                  // [kTb][kTb + 1]
  double* Bs = As + kTb * kPitch;          // [kTb][kTb + 1]
  const int tid = threadIdx.x, tx = tid % 16, ty = tid / 16;
  const int per = a.npairs * a.nchunk;
  for (int item = blockIdx.x; item < nact * per; item += gridDim.x) {
    const CqProb& P = a.prob[act[item / per]];
    const double* __restrict__ X = pass == 0 ? P.Y : P.Q;
    const int local = item % per;
    const int pair = local % a.npairs, chunk = local / a.npairs;
    int bi, bj;
    pair_of(pair, a.T, bi, bj);
    const int r0 = chunk * a.chunk_rows;
    const int r1 = min(a.rows, r0 + a.chunk_rows);
    double acc00 = 0.0, acc01 = 0.0, acc10 = 0.0, acc11 = 0.0;
    for (int rs = r0; rs < r1; rs += kTb) {
      __syncthreads();
      for (int e = tid; e < kTb * kTb; e += kCqThreads) {
        const int rr = e / kTb, cc = e % kTb;
        const int r = rs + rr, ci = bi * kTb + cc, cj = bj * kTb + cc;
        As[rr * kPitch + cc] = (r < r1 && ci < a.n) ? X[(long long)r * a.n + ci] : 0.0;
        Bs[rr * kPitch + cc] = (r < r1 && cj < a.n) ? X[(long long)r * a.n + cj] : 0.0;
      }
      __syncthreads();
#pragma unroll 8
      for (int rr = 0; rr < kTb; ++rr) {
        const double a0 = As[rr * kPitch + 2 * ty], a1 = As[rr * kPitch + 2 * ty + 1];
        const double b0 = Bs[rr * kPitch + 2 * tx], b1 = Bs[rr * kPitch + 2 * tx + 1];
        acc00 = fma(a0, b0, acc00);
        acc01 = fma(a0, b1, acc01);
        acc10 = fma(a1, b0, acc10);
        acc11 = fma(a1, b1, acc11);
      }
    }
    double* out = P.part + ((long long)chunk * a.npairs + pair) * (kTb * kTb);
    out[(2 * ty) * kTb + 2 * tx] = acc00;
    out[(2 * ty) * kTb + 2 * tx + 1] = acc01;
    out[(2 * ty + 1) * kTb + 2 * tx] = acc10;
    out[(2 * ty + 1) * kTb + 2 * tx + 1] = acc11;
  }
}

__device__ __forceinline__ double gram_entry(const CqArgs& a, const CqProb& P, int i,
                                             int j) {  // any i, j
  if (i > j) {
    const int t = i;
    i = j;
    j = t;
  }
  const int bi = i / kTb, bj = j / kTb;
  const long long off =
      (long long)pair_index(bi, bj, a.T) * (kTb * kTb) + (i % kTb) * kTb + (j % kTb);
  double s = 0.0;
  for (int c = 0; c < a.nchunk; ++c) s += P.part[(long long)c * a.npairs * (kTb * kTb) + off];
  return s;
}

// Phase R: G' (lower triangle) = D^-1 G D^-1 + shift I, D, max |G' - I| and
// ||G' - I||_F^2, for every active problem.
__device__ void reduce_scale(const CqArgs& a, double shift, int pass, const int* act, int nact) {
  const long long nn = (long long)a.n * a.n;
  for (int ia = 0; ia < nact; ++ia) {
    const CqProb& P = a.prob[act[ia]];
    double local = 0.0, sq = 0.0;
    for (long long e = blockIdx.x * (long long)kCqThreads + threadIdx.x; e < nn;
         e += (long long)gridDim.x * kCqThreads) {
      const int i = (int)(e / a.n), j = (int)(e % a.n);
      if (j > i) continue;
      const double gii = gram_entry(a, P, i, i), gjj = gram_entry(a, P, j, j);
      const double di = gii > 0.0 ? sqrt(gii) : 1.0, dj = gjj > 0.0 ? sqrt(gjj) : 1.0;
      double v = gram_entry(a, P, i, j) / (di * dj);
      if (i == j) {
        v += shift;
        P.dscale[i] = di;
        P.dinv[i] = 1.0 / di;
      }
      P.G[(long long)i * a.n + j] = v;
      const double dev = v - (i == j ? 1.0 : 0.0);
      local = fmax(local, fabs(dev));
      sq = fma(i == j ? 1.0 : 2.0, dev * dev, sq);  // G' - I is symmetric
    }
    for (int o = 16; o > 0; o >>= 1) {
      local = fmax(local, __shfl_xor_sync(0xffffffffu, local, o));
      sq += __shfl_xor_sync(0xffffffffu, sq, o);
    }
    if ((threadIdx.x & 31) == 0 && local > 0.0)
      atomicMax(reinterpret_cast<unsigned long long*>(P.emax + pass),
                (unsigned long long)__double_as_longlong(local));
    if ((threadIdx.x & 31) == 0 && sq > 0.0) atomicAdd(P.fro2 + pass, sq);
  }
}

// 1 / sqrt(d) for d in [1e-30, 1e30] (every pivot of a scaled Gram): the FP32
// hardware estimate refined by two Newton-Raphson steps for the reciprocal
// square root, y <- y + y (1 - d y^2) / 2, whose error squares at each step
// (2^-22 -> 2^-44 -> below FP64 rounding).  On the pivot chain of the Cholesky
// this replaces an FP64 square root and a division.
__device__ __forceinline__ double cq_rsqrt(double d) {
  double y = (double)rsqrtf((float)d);
#pragma unroll
  for (int i = 0; i < 2; ++i) {
    const double r = fma(-d * y, y, 1.0);
    y = fma(0.5 * y, r, y);
  }
  return y;
}

// Diagonal block p: Cholesky (lower) and its inverse into Linv[p] by one CTA.
// GB300 retires well under one FP64 warp-instruction per clock per SM
// sub-partition, so what sets this phase's length is the chain of 32 pivots
// and the FP64 instructions queued beside it.  Thread 0 (warp 0) only runs the
// pivot chain, one step ahead: while the other warps apply step k, it updates
// the next diagonal entry and takes its reciprocal square root.  Warps 1-3 and
// 5-7 (the sub-partitions warp 0 does not use) apply step k: column k of the
// factor, the rank-1 update of the trailing triangle of the working copy Lm,
// and the same elimination on the rows of X, which starts as the identity and
// ends as L^-1 (Gauss-Jordan on the unit matrix; row k's own scaling by
// 1 / L_kk is applied once at the end).  One barrier per step.  Pivot rules:
// shifted pass -> floor at `floor` (counted); unshifted passes -> a pivot
// <= tau marks a dependent column (its L column is e_k).
__device__ __forceinline__ void cq_pivot(const CqArgs& a, const CqProb& P, int col, double d,
                                         double floor, double tau, bool use_mask, double* s_d,
                                         double* s_y, int* s_dep, int k) {
  int dep = 0;
  if (use_mask && !(d > tau)) {  // column lies in the span of the earlier ones
    dep = 1;
    d = 1.0;
    P.defmask[col] = 1;
  } else if (!(d > floor)) {
    d = floor;
    atomicAdd(a.floored, 1);
  }
  s_d[k] = d;
  s_y[k] = cq_rsqrt(d);
  s_dep[k] = dep;
}

__device__ void diag_factor(const CqArgs& a, const CqProb& P, int p, double floor, double tau,
                            bool use_mask) {
  double* Lm = cq_smem();                  // [kTb][kTb + 1] working copy
  double* Lo = Lm + kTb * kPitch;          // [kTb][kTb + 1] the factor
  double* Xm = Lo + kTb * kPitch;          // [kTb][kTb + 1] its inverse
  double* s_d = Xm + kTb * kPitch;         // [kTb] pivots after the rules
  double* s_y = s_d + kTb;                 // [kTb] 1 / sqrt(pivot)
  __shared__ int s_dep[kTb];
  const int t = threadIdx.x, warp = t / 32;
  const int j0 = p * kTb, jb = min(kTb, a.n - j0);
  // workers: warps not on warp 0's sub-partition
  const bool worker = (warp % 4) != 0;
  const int wid = (warp / 4) * 96 + (warp % 4 - 1) * 32 + t % 32;  // 0 .. 191
  constexpr int kWorkers = kCqThreads / 4 * 3;
  __syncthreads();
  for (int e = t; e < kTb * kTb; e += kCqThreads) {
    const int i = e / kTb, j = e % kTb;
    Lm[i * kPitch + j] = (i < jb && j < jb && j <= i) ? P.G[(long long)(j0 + i) * a.n + j0 + j] : 0.0;
    Lo[i * kPitch + j] = 0.0;
    Xm[i * kPitch + j] = (i == j && i < jb) ? 1.0 : 0.0;
  }
  __syncthreads();
  if (t == 0) cq_pivot(a, P, j0, Lm[0], floor, tau, use_mask, s_d, s_y, s_dep, 0);
  __syncthreads();
  for (int k = 0; k < jb; ++k) {
    const double y = s_y[k];
    const bool dep = s_dep[k] != 0;
    const int m = jb - k - 1;  // rows below the pivot
    if (t == 0) {
      Lo[k * kPitch + k] = s_d[k] * y;
      if (m > 0) {
        double d1 = Lm[(k + 1) * kPitch + k + 1];
        if (!dep) {
          const double l = Lm[(k + 1) * kPitch + k] * y;
          d1 = fma(-l, l, d1);
        }
        cq_pivot(a, P, j0 + k + 1, d1, floor, tau, use_mask, s_d, s_y, s_dep, k + 1);
      }
    } else if (worker) {
      const double y2 = y * y;
      const int ntri = m * (m + 1) / 2;  // (i, j), k < j <= i < jb; entry 0 is the next pivot
      const int nx = m * (k + 1);        // (i, c), k < i < jb, c <= k
      for (int e = wid; e < ntri + nx + m; e += kWorkers) {
        if (e < ntri) {
          if (e == 0 || dep) continue;
          int r = (int)((sqrtf(8.0f * (float)e + 1.0f) - 1.0f) * 0.5f);
          if (r * (r + 1) / 2 > e) --r;
          if ((r + 1) * (r + 2) / 2 <= e) ++r;
          const int i = k + 1 + r, j = k + 1 + (e - r * (r + 1) / 2);
          Lm[i * kPitch + j] = fma(-Lm[i * kPitch + k] * y2, Lm[j * kPitch + k], Lm[i * kPitch + j]);
        } else if (e < ntri + nx) {
          if (dep) continue;
          const int e2 = e - ntri;
          const int i = k + 1 + e2 / (k + 1), c = e2 % (k + 1);
          Xm[i * kPitch + c] = fma(-Lm[i * kPitch + k] * y2, Xm[k * kPitch + c], Xm[i * kPitch + c]);
        } else {
          const int i = k + 1 + (e - ntri - nx);
          Lo[i * kPitch + k] = dep ? 0.0 : Lm[i * kPitch + k] * y;
        }
      }
    }
    __syncthreads();
  }
  for (int e = t; e < kTb * kTb; e += kCqThreads) {
    const int i = e / kTb, j = e % kTb;
    if (i < jb && j < jb) P.G[(long long)(j0 + i) * a.n + j0 + j] = Lo[i * kPitch + j];
    P.Linv[(long long)p * kTb * kTb + e] = (i < jb && j <= i) ? Xm[i * kPitch + j] * s_y[i] : 0.0;
  }
}

// Panel p: L_ip = G'_ip Linv_pp^T for block rows i > p of every problem that
// takes the Cholesky (chol[q]); items are 8-row groups.
__device__ void panel_solve(const CqArgs& a, int p, const bool* chol) {
  double* Li = cq_smem();                  // [kTb][kTb + 1]
  double* Gr = Li + kTb * kPitch;          // [8][kTb + 1]
  const int tid = threadIdx.x;
  const int j0 = p * kTb, jb = min(kTb, a.n - j0);
  const int r_lo = j0 + jb;
  const int groups = (a.n - r_lo + 7) / 8;
  for (int item = blockIdx.x; item < a.nprob * groups; item += gridDim.x) {
    const int q = item / groups;
    if (!chol[q]) continue;
    const CqProb& P = a.prob[q];
    const int r0 = r_lo + (item % groups) * 8;
    __syncthreads();
    for (int e = tid; e < kTb * kTb; e += kCqThreads)
      Li[(e / kTb) * kPitch + e % kTb] = P.Linv[(long long)p * kTb * kTb + e];
    {
      const int rr = tid / kTb, cc = tid % kTb;
      const int r = r0 + rr;
      Gr[rr * kPitch + cc] = (r < a.n && cc < jb) ? P.G[(long long)r * a.n + j0 + cc] : 0.0;
    }
    __syncthreads();
    const int rr = tid / kTb, cc = tid % kTb;
    double acc = 0.0;
#pragma unroll 8
    for (int k = 0; k < kTb; ++k) acc = fma(Gr[rr * kPitch + k], Li[cc * kPitch + k], acc);
    const int r = r0 + rr;
    if (r < a.n && cc < jb) P.G[(long long)r * a.n + j0 + cc] = acc;
  }
}

// Trailing update after panel p: G'_ij -= L_ip L_jp^T for p < bj <= bi (block
// coordinates), lower blocks only; items are (problem, block pair, 8-row group).
__device__ void trailing_update(const CqArgs& a, int p, const bool* chol) {
  double* Lj = cq_smem();                  // [kTb][kTb + 1]
  double* Lr = Lj + kTb * kPitch;          // [8][kTb + 1]
  const int tid = threadIdx.x;
  const int j0 = p * kTb, jb = min(kTb, a.n - j0);
  const int nb = a.T - p - 1;  // remaining block rows/cols
  const int pairs = nb * (nb + 1) / 2;
  const int per = pairs * 4;
  for (int item = blockIdx.x; item < a.nprob * per; item += gridDim.x) {
    const int q = item / per;
    if (!chol[q]) continue;
    const CqProb& P = a.prob[q];
    const int local = item % per;
    const int pr = local / 4, g = local % 4;
    int ci, cj;  // ci <= cj in 0..nb-1 : block col = p+1+ci, block row = p+1+cj
    pair_of(pr, nb, ci, cj);
    const int bc = p + 1 + ci, br = p + 1 + cj;
    const int r0 = br * kTb + g * 8;
    __syncthreads();
    for (int e = tid; e < kTb * kTb; e += kCqThreads) {
      const int rr = e / kTb, kk = e % kTb;
      const int r = bc * kTb + rr;
      Lj[rr * kPitch + kk] = (r < a.n && kk < jb) ? P.G[(long long)r * a.n + j0 + kk] : 0.0;
    }
    {
      const int rr = tid / kTb, kk = tid % kTb;
      const int r = r0 + rr;
      Lr[rr * kPitch + kk] = (r < a.n && kk < jb) ? P.G[(long long)r * a.n + j0 + kk] : 0.0;
    }
    __syncthreads();
    const int rr = tid / kTb, cc = tid % kTb;
    const int r = r0 + rr, col = bc * kTb + cc;
    if (r < a.n && col < a.n && col <= r) {
      double acc = 0.0;
#pragma unroll 8
      for (int k = 0; k < kTb; ++k) acc = fma(Lr[rr * kPitch + k], Lj[cc * kPitch + k], acc);
      P.G[(long long)r * a.n + col] -= acc;
    }
  }
}

// Phase T: Q = X D^-1 L^-T (full) or Q = X D^-1 (I - U) (near identity) for the
// 16-row blocks this CTA owns; then, when asked, flagged columns become Gaussian.
__device__ void substitute(const CqArgs& a, int pass, const bool* near_ids, const bool* refills,
                           const bool* scale_only, unsigned long long seed, const int* act,
                           int nact) {
  double* Xs = cq_smem();                  // [kRowBlock][n] scaled input rows
  double* Qs = Xs + kRowBlock * a.n;       // [kRowBlock][n] output rows
  double* Lt = Qs + kRowBlock * a.n;       // [kTb][kTb + 1] a tile of L (or U^T)
  double* Tt = Lt + kTb * kPitch;          // [kRowBlock][kTb + 1]
  const int tid = threadIdx.x;
  const int nblk = (a.rows + kRowBlock - 1) / kRowBlock;
  for (int item = blockIdx.x; item < nact * nblk; item += gridDim.x) {
    const int q = act[item / nblk];
    const CqProb& P = a.prob[q];
    const double* __restrict__ X = pass == 0 ? P.Y : P.Q;
    const bool near_id = near_ids[q], refill = refills[q];
    const int r0 = (item % nblk) * kRowBlock;
    if (scale_only[q]) {  // orthonormal input: Q = X D^-1, element by element
      for (int e = tid; e < kRowBlock * a.n; e += kCqThreads) {
        const int r = r0 + e / a.n, cc = e % a.n;
        if (r < a.rows) P.Q[(long long)r * a.n + cc] = X[(long long)r * a.n + cc] * P.dinv[cc];
      }
      continue;
    }
    __syncthreads();
    for (int e = tid; e < kRowBlock * a.n; e += kCqThreads) {
      const int rr = e / a.n, cc = e % a.n;
      const int r = r0 + rr;
      Xs[e] = r < a.rows ? X[(long long)r * a.n + cc] * P.dinv[cc] : 0.0;
    }
    __syncthreads();
    for (int p = 0; p < a.T; ++p) {
      const int j0 = p * kTb, jb = min(kTb, a.n - j0);
      // thread -> (row rr, col cc) of the 16 x 32 panel block, two per thread
      const int cc = tid % kTb, rr0 = tid / kTb;  // rows rr0 and rr0 + 8
      double acc0 = 0.0, acc1 = 0.0;
      const double* src = near_id ? Xs : Qs;
      for (int k0 = 0; k0 < j0; k0 += kTb) {
        __syncthreads();
        for (int e = tid; e < kTb * kTb; e += kCqThreads) {
          const int i = e / kTb, k = e % kTb;  // Lt[(i) * kPitch + (k)] = L[j0 + i][k0 + k]
          Lt[(i) * kPitch + (k)] = (i < jb) ? P.G[(long long)(j0 + i) * a.n + k0 + k] : 0.0;
        }
        __syncthreads();
#pragma unroll 8
        for (int k = 0; k < kTb; ++k) {
          const double l = Lt[(cc) * kPitch + (k)];
          acc0 = fma(src[rr0 * a.n + k0 + k], l, acc0);
          acc1 = fma(src[(rr0 + 8) * a.n + k0 + k], l, acc1);
        }
      }
      if (near_id) {
        // Q_j = xs_j - sum_{k < j} xs_k E_jk, including k inside this panel
        __syncthreads();
        for (int e = tid; e < kTb * kTb; e += kCqThreads) {
          const int i = e / kTb, k = e % kTb;
          Lt[(i) * kPitch + (k)] = (i < jb && k < i) ? P.G[(long long)(j0 + i) * a.n + j0 + k] : 0.0;
        }
        __syncthreads();
        for (int k = 0; k < kTb; ++k) {
          const double l = Lt[(cc) * kPitch + (k)];
          acc0 = fma(Xs[rr0 * a.n + j0 + k], l, acc0);
          acc1 = fma(Xs[(rr0 + 8) * a.n + j0 + k], l, acc1);
        }
        if (cc < jb) {
          Qs[rr0 * a.n + j0 + cc] = Xs[rr0 * a.n + j0 + cc] - acc0;
          Qs[(rr0 + 8) * a.n + j0 + cc] = Xs[(rr0 + 8) * a.n + j0 + cc] - acc1;
        }
      } else {
        // T = xs_panel - Q_{<p} L_{p,<p}^T, then Q_panel = T Linv_pp^T
        Tt[(rr0) * kPitch + (cc)] = cc < jb ? Xs[rr0 * a.n + j0 + cc] - acc0 : 0.0;
        Tt[(rr0 + 8) * kPitch + (cc)] = cc < jb ? Xs[(rr0 + 8) * a.n + j0 + cc] - acc1 : 0.0;
        __syncthreads();
        for (int e = tid; e < kTb * kTb; e += kCqThreads)
          Lt[(e / kTb) * kPitch + (e % kTb)] = P.Linv[(long long)p * kTb * kTb + e];
        __syncthreads();
        double q0 = 0.0, q1 = 0.0;
#pragma unroll 8
        for (int k = 0; k < kTb; ++k) {
          const double l = Lt[(cc) * kPitch + (k)];
          q0 = fma(Tt[(rr0) * kPitch + (k)], l, q0);
          q1 = fma(Tt[(rr0 + 8) * kPitch + (k)], l, q1);
        }
        if (cc < jb) {
          Qs[rr0 * a.n + j0 + cc] = q0;
          Qs[(rr0 + 8) * a.n + j0 + cc] = q1;
        }
      }
      __syncthreads();
    }
    for (int e = tid; e < kRowBlock * a.n; e += kCqThreads) {
      const int rr = e / a.n, cc = e % a.n;
      const int r = r0 + rr;
      if (r >= a.rows) continue;
      double v = Qs[e];
      if (refill && P.defmask[cc])
        v = cq_gauss(seed, (unsigned long long)cc * a.rows + r);
      P.Q[(long long)r * a.n + cc] = v;
    }
  }
}

__device__ bool cholqr_passes(const CqArgs& a, double u);

constexpr int kCqMaxStamps = 512;

// Diagnostics: block 0 records the global timer after each grid barrier.
__device__ __forceinline__ void cq_stamp(const CqArgs& a, int tag) {
  if (!a.stamps || blockIdx.x != 0 || threadIdx.x != 0) return;
  const unsigned long long k = a.stamps[0];
  if (k >= kCqMaxStamps) return;
  unsigned long long t;
  asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
  a.stamps[1 + 2 * k] = (unsigned long long)tag;
  a.stamps[2 + 2 * k] = t;
  a.stamps[0] = k + 1;
}

__global__ void __launch_bounds__(kCqThreads, 1) cholqr_kernel(CqArgs a) {
  const double u = 1.1102230246251565e-16;
  const bool ok = cholqr_passes(a, u);
  if (!ok && blockIdx.x == 0 && threadIdx.x == 0 && a.err_out) atomicExch(a.err_out, 1);
}

__device__ bool cholqr_passes(const CqArgs& a, double u) {
  __shared__ bool s_chol[kCqMaxProb], s_near[kCqMaxProb], s_refill[kCqMaxProb],
      s_scale[kCqMaxProb], s_last[kCqMaxProb];
  __shared__ int s_act[kCqMaxProb], s_nact;
  double flops = 0.0;  // block 0, thread 0: flops of the passes run
  const double gram = (double)a.rows * a.n * a.n, chol = (double)a.n * a.n * a.n / 3.0;
  if (threadIdx.x == 0) {
    for (int q = 0; q < a.nprob; ++q) s_act[q] = q;
    s_nact = a.nprob;
  }
  __syncthreads();
  cq_stamp(a, 0);
  for (int pass = 0; pass < a.passes && s_nact > 0; ++pass) {
    const bool shift_pass = pass == 0 && a.shifted;
    gram_partials(a, pass, s_act, s_nact);
    if (!cq_barrier(a.fl)) return false;
    cq_stamp(a, 1);
    // the masks of the previous pass have been read by every block by now
    for (int q = 0; q < a.nprob; ++q)
      for (int j = blockIdx.x * kCqThreads + threadIdx.x; j < a.n; j += gridDim.x * kCqThreads)
        a.prob[q].defmask[j] = 0;
    const double shift =
        shift_pass ? 11.0 * ((double)a.rows * a.n + (double)a.n * (a.n + 1)) * u * a.n : 0.0;
    reduce_scale(a, shift, pass, s_act, s_nact);
    if (!cq_barrier(a.fl)) return false;
    cq_stamp(a, 2);
    // every block must take the same branches (the barrier count depends on them):
    // thread 0 reads each reduced maximum with an acquire load and broadcasts it
    if (threadIdx.x == 0) {
      for (int q = 0; q < a.nprob; ++q) {
        s_near[q] = s_chol[q] = s_refill[q] = s_scale[q] = s_last[q] = false;
      }
      for (int ia = 0; ia < s_nact; ++ia) {
        const int q = s_act[ia];
        unsigned long long bits, fbits;
        asm volatile("ld.acquire.gpu.global.u64 %0, [%1];"
                     : "=l"(bits)
                     : "l"(a.prob[q].emax + pass)
                     : "memory");
        asm volatile("ld.acquire.gpu.global.u64 %0, [%1];"
                     : "=l"(fbits)
                     : "l"(a.prob[q].fro2 + pass)
                     : "memory");
        const double e = __longlong_as_double((long long)bits);
        const double f2 = __longlong_as_double((long long)fbits);
        s_near[q] = !shift_pass && e < kNearIdentity;
        s_scale[q] = !shift_pass && e < kOrthonormal;
        s_chol[q] = !s_near[q];
        s_last[q] = !shift_pass && (s_scale[q] || f2 <= kLastPassFro * kLastPassFro);
        s_refill[q] = !s_near[q] && !s_last[q] && pass > 0 && pass + 1 < a.passes;
        flops += s_scale[q] ? gram : 2.0 * gram + (s_chol[q] ? chol : 0.0);
      }
    }
    __syncthreads();
    bool any_chol = false;
    for (int q = 0; q < a.nprob; ++q) any_chol = any_chol || s_chol[q];
    if (any_chol) {
      for (int p = 0; p < a.T; ++p) {
        if (blockIdx.x < a.nprob && s_chol[blockIdx.x])  // inactive problems: s_chol false
          diag_factor(a, a.prob[blockIdx.x], p, 1e-28, 1e-12, !shift_pass && pass > 0);
        if (!cq_barrier(a.fl)) return false;
        cq_stamp(a, 3);
        panel_solve(a, p, s_chol);
        if (!cq_barrier(a.fl)) return false;
        cq_stamp(a, 4);
        if (p + 1 < a.T) {
          trailing_update(a, p, s_chol);
          if (!cq_barrier(a.fl)) return false;
          cq_stamp(a, 5);
        }
      }
    }
    substitute(a, pass, s_near, s_refill, s_scale, a.seed + (unsigned long long)pass, s_act,
               s_nact);
    if (!cq_barrier(a.fl)) return false;
    cq_stamp(a, 6);
    // problems whose pass was their last leave the active list (same in every block)
    if (threadIdx.x == 0) {
      int n = 0;
      for (int ia = 0; ia < s_nact; ++ia)
        if (!s_last[s_act[ia]]) s_act[n++] = s_act[ia];
      s_nact = n;
    }
    __syncthreads();
  }
  if (blockIdx.x == 0 && threadIdx.x == 0 && a.flops_out) atomicAdd(a.flops_out, flops);
  return true;
}

// Work layout (doubles): Gram partials | G' (n x n) | diagonal-block inverses |
// D | D^-1 | max |G' - I| per pass (8) | ||G' - I||_F^2 per pass (8) |
// dependent-column mask (n ints) | barrier words.
void cholqr_layout(int rows, int n, int nsm, int& T, int& npairs, int& nchunk, int& chunk_rows) {
  T = (n + kTb - 1) / kTb;
  npairs = T * (T + 1) / 2;
  nchunk = (2 * nsm + npairs - 1) / npairs;
  const int max_chunks = (rows + kTb - 1) / kTb;
  if (nchunk > max_chunks) nchunk = max_chunks;
  if (nchunk < 1) nchunk = 1;
  chunk_rows = ((rows + nchunk - 1) / nchunk + kTb - 1) / kTb * kTb;
  nchunk = (rows + chunk_rows - 1) / chunk_rows;
}

int cholqr_sm_count() {
  int dev = 0, nsm = 0;
  if (cudaGetDevice(&dev) != cudaSuccess ||
      cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess)
    return 0;
  return nsm;
}

}  // namespace

// doubles of one problem's part of the work buffer
size_t cholqr_prob_doubles(int rows, int n) {
  const int nsm = cholqr_sm_count();
  int T, npairs, nchunk, chunk_rows;
  cholqr_layout(rows, n, nsm > 0 ? nsm : 1, T, npairs, nchunk, chunk_rows);
  return (size_t)nchunk * npairs * kTb * kTb + (size_t)n * n + (size_t)T * kTb * kTb + 2 * n + 16 +
         (size_t)(n + 1) / 2;
}

size_t cholqr_work_doubles(int rows, int n, int nprob) {
  return (size_t)nprob * cholqr_prob_doubles(rows, n) + 8;
}

int cholqr_fused_batch(cudaStream_t s, int nprob, const double* const* Y, double* const* Q,
                       int rows, int n, int passes, bool shifted, double* work, int* err_word,
                       int* floored, double* flops_out, unsigned long long seed,
                       long long* launches, cudaEvent_t t0, cudaEvent_t t1) {
  if (nprob < 1 || nprob > kCqMaxProb || n < 1 || n > kCqMaxN || rows < 1 || passes < 1 ||
      passes > 8)
    return -1;
  const int nsm = cholqr_sm_count();
  if (nsm < 1) return -3;
  CqArgs a;
  a.nprob = nprob;
  a.rows = rows;
  a.n = n;
  a.passes = passes;
  a.shifted = shifted ? 1 : 0;
  cholqr_layout(rows, n, nsm, a.T, a.npairs, a.nchunk, a.chunk_rows);
  const size_t per = cholqr_prob_doubles(rows, n);
  for (int q = 0; q < nprob; ++q) {
    CqProb& P = a.prob[q];
    P.Y = Y[q];
    P.Q = Q[q];
    double* w = work + (size_t)q * per;
    P.part = w;
    w += (size_t)a.nchunk * a.npairs * kTb * kTb;
    P.G = w;
    w += (size_t)n * n;
    P.Linv = w;
    w += (size_t)a.T * kTb * kTb;
    P.dscale = w;
    w += n;
    P.dinv = w;
    w += n;
    P.emax = w;
    P.fro2 = w + 8;
    w += 16;
    P.defmask = reinterpret_cast<int*>(w);
    if (cudaMemsetAsync(P.emax, 0, 16 * sizeof(double), s) != cudaSuccess) return -3;
  }
  a.fl = reinterpret_cast<DevFlags*>(work + (size_t)nprob * per);
  static_assert(sizeof(DevFlags) <= 8 * sizeof(double), "DevFlags must fit its slot");
  a.err_out = err_word;
  a.floored = floored;
  a.flops_out = flops_out;
  a.stamps = cq_stamps_buffer();
  a.seed = seed;
  const size_t dyn = sizeof(double) * cq_smem_doubles(n);
  static int attr_dev = -1;
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess) return -3;
  if (attr_dev != dev) {
    if (cudaFuncSetAttribute(cholqr_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                             (int)(sizeof(double) * cq_smem_doubles(kCqMaxN))) != cudaSuccess)
      return -3;
    attr_dev = dev;
  }
  int per_sm = 0;
  if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, cholqr_kernel, kCqThreads, dyn) !=
          cudaSuccess ||
      per_sm < 1)
    return -3;
  if (per_sm > 2) per_sm = 2;
  // this launch's barrier words start at zero
  if (cudaMemsetAsync(a.fl, 0, sizeof(DevFlags), s) != cudaSuccess) return -3;
  void* args[] = {&a};
  if (launch_cooperative(reinterpret_cast<const void*>(cholqr_kernel), dim3(nsm * per_sm),
                         dim3(kCqThreads), args, dyn, s, t0, t1) != cudaSuccess)
    return -3;
  ++*launches;
  return 0;
}

// CTM_TRACE=3: a device buffer of phase timestamps for the next launches.
namespace {
unsigned long long* g_stamps = nullptr;
}
unsigned long long* cq_stamps_buffer() {
  static int on = -1;
  if (on < 0) {
    const char* e = std::getenv("CTM_TRACE");
    on = (e && *e == '3') ? 1 : 0;
  }
  if (!on) return nullptr;
  if (!g_stamps && cudaMalloc(&g_stamps, sizeof(unsigned long long) * (1 + 2 * kCqMaxStamps)) != cudaSuccess)
    g_stamps = nullptr;
  if (g_stamps) cudaMemset(g_stamps, 0, sizeof(unsigned long long));
  return g_stamps;
}

int cholqr_read_stamps(cudaStream_t s, double* ms_by_tag /* [8] */) {
  if (!g_stamps) return -1;
  if (cudaStreamSynchronize(s) != cudaSuccess) return -3;
  std::vector<unsigned long long> h(1 + 2 * kCqMaxStamps);
  if (cudaMemcpy(h.data(), g_stamps, sizeof(unsigned long long) * h.size(), cudaMemcpyDeviceToHost) != cudaSuccess)
    return -3;
  for (int t = 0; t < 8; ++t) ms_by_tag[t] = 0.0;
  const unsigned long long k = h[0] < (unsigned long long)kCqMaxStamps ? h[0] : kCqMaxStamps;
  for (unsigned long long i = 1; i < k; ++i) {
    const int tag = (int)h[1 + 2 * i];
    ms_by_tag[tag & 7] += 1e-6 * (double)(h[2 + 2 * i] - h[2 * i]);
  }
  return 0;
}

int cholqr_read_emax(cudaStream_t s, const double* work, int rows, int n, int nprob, double* out) {
  const int nsm = cholqr_sm_count();
  if (nsm < 1 || nprob < 1 || nprob > kCqMaxProb) return -1;
  int T, npairs, nchunk, chunk_rows;
  cholqr_layout(rows, n, nsm, T, npairs, nchunk, chunk_rows);
  const size_t off =
      (size_t)nchunk * npairs * kTb * kTb + (size_t)n * n + (size_t)T * kTb * kTb + 2 * (size_t)n;
  const size_t per = cholqr_prob_doubles(rows, n);
  if (cudaStreamSynchronize(s) != cudaSuccess) return -3;
  for (int q = 0; q < nprob; ++q)
    if (cudaMemcpy(out + 16 * q, work + q * per + off, 16 * sizeof(double), cudaMemcpyDeviceToHost) !=
        cudaSuccess)
      return -3;
  return 0;
}

int cholqr_fused(cudaStream_t s, const double* Y, double* Q, int rows, int n, int passes,
                 bool shifted, double* work, int* err_word, int* floored, double* flops_out,
                 unsigned long long seed, long long* launches, cudaEvent_t t0, cudaEvent_t t1) {
  return cholqr_fused_batch(s, 1, &Y, &Q, rows, n, passes, shifted, work, err_word, floored,
                            flops_out, seed, launches, t0, t1);
}

}  // namespace ctm
