// FP64 dense linear algebra for the projector factorisations: one-sided
// (Hestenes) Jacobi SVD with a parallel round-robin ordering, sorting and
// gathering of singular vectors, Frobenius normalisation, and a counter-based
// Gaussian generator for randomized range finding.
//
// Methods: one-sided Jacobi with the Rutishauser rotation and the
// cosine-based stopping rule (Demmel & Veselic, SIAM J. Matrix Anal. Appl. 13,
// 1204 (1992)); round-robin ("chess tournament") pair ordering (Brent & Luk,
// SIAM J. Sci. Stat. Comput. 6, 69 (1985)); SplitMix64 (Steele, Lea & Flood,
// OOPSLA 2014) with the Box-Muller transform.
#include "ctm_internal.h"

#include <cmath>
#include <cstddef>
#include <mutex>

namespace ctm {

static_assert(offsetof(DevFlags, error) == kDevFlagsResetBytes, "DevFlags layout");

// ---------------------------------------------------------------------------
// Bounded grid barrier for cooperative launches.  Every wait has an iteration
// cap; on timeout the kernel records an error and all blocks return.
// ---------------------------------------------------------------------------
constexpr long long kBarrierCycleLimit = 4000000000ll;  // ~2 s of SM clock

__device__ __forceinline__ unsigned ld_acquire_u32(const unsigned* p) {
  unsigned v;
  asm volatile("ld.acquire.gpu.global.u32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
  return v;
}

__device__ __forceinline__ unsigned atom_add_release_u32(unsigned* p, unsigned v) {
  unsigned old;
  asm volatile("atom.add.release.gpu.global.u32 %0, [%1], %2;" : "=r"(old) : "l"(p), "r"(v)
               : "memory");
  return old;
}

// Sense-by-generation grid barrier: one release-add per block, the last block
// resets the counter and bumps the generation, the others poll the generation
// with acquire loads.  The poll gives up after kBarrierCycleLimit clocks.
__device__ __forceinline__ bool grid_barrier(DevFlags* fl, unsigned nblocks) {
  __shared__ int s_ok;
  __syncthreads();
  if (threadIdx.x == 0) {
    const unsigned g = ld_acquire_u32(&fl->bar_gen);
    const unsigned arrived = atom_add_release_u32(&fl->bar_count, 1u);
    if (arrived == nblocks - 1) {
      atomicExch(&fl->bar_count, 0u);
      atom_add_release_u32(&fl->bar_gen, 1u);
    } else {
      const long long t0 = clock64();
      while (ld_acquire_u32(&fl->bar_gen) == g) {
        if (clock64() - t0 > kBarrierCycleLimit) {
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

template <int NT>
__device__ __forceinline__ void block_sum3(double& a, double& b, double& c) {
  __shared__ double red[3][NT / 32];
  for (int o = 16; o > 0; o >>= 1) {
    a += __shfl_xor_sync(0xffffffffu, a, o);
    b += __shfl_xor_sync(0xffffffffu, b, o);
    c += __shfl_xor_sync(0xffffffffu, c, o);
  }
  const int w = threadIdx.x / 32, l = threadIdx.x % 32;
  __syncthreads();
  if (l == 0) {
    red[0][w] = a;
    red[1][w] = b;
    red[2][w] = c;
  }
  __syncthreads();
  a = b = c = 0.0;
  for (int i = 0; i < NT / 32; ++i) {  // fixed order: deterministic
    a += red[0][i];
    b += red[1][i];
    c += red[2][i];
  }
}

constexpr int kJacobiThreads = 256;
constexpr int kWarpJacobiMaxRows = 4096;  // warp-per-pair Jacobi up to this column length

// Column held at round-robin position p during step s (n even, position 0 fixed).
__device__ __forceinline__ int rr_col(int p, int s, int n) {
  return p == 0 ? 0 : 1 + (p - 1 + s) % (n - 1);
}

__global__ void __launch_bounds__(kJacobiThreads)
jacobi_kernel(double* __restrict__ Xall, int nrows, int ncols, int npad, double* __restrict__ V,
              DevFlags* fl, int max_sweeps, double tol, int nprob, long long pstride,
              double tiny_rel) {
  const unsigned nblocks = gridDim.x;
  const int npairs = npad / 2;
  double* X = Xall;
  // columns whose squared norm is below tiny_rel ||X||_F^2 lie under the
  // resolution that matters (1e-32: FP64; 1e-24 when only singular values
  // above 1e-12 of the largest are wanted): they are still rotated but do not
  // count for convergence
  {
    double part = 0.0, z1 = 0.0, z2 = 0.0;
    const long long per = (long long)nrows * ncols;
    for (int p = 0; p < nprob; ++p)
      for (long long e = blockIdx.x * (long long)kJacobiThreads + threadIdx.x; e < per;
           e += (long long)gridDim.x * kJacobiThreads)
        part = fma(Xall[p * pstride + e], Xall[p * pstride + e], part);
    block_sum3<kJacobiThreads>(part, z1, z2);
    if (threadIdx.x == 0 && part > 0.0) atomicAdd(&fl->fro2, part);
    if (!grid_barrier(fl, nblocks)) return;
  }
  const double tiny = tiny_rel * (*(volatile double*)&fl->fro2);
  for (int sweep = 0; sweep < max_sweeps; ++sweep) {
    double local_max = 0.0;
    for (int step = 0; step < npad - 1; ++step) {
      for (int kk = blockIdx.x; kk < npairs * nprob; kk += gridDim.x) {
        const int k = kk % npairs;
        X = Xall + (long long)(kk / npairs) * pstride;
        int i = rr_col(k, step, npad);
        int j = rr_col(npad - 1 - k, step, npad);
        if (i >= ncols || j >= ncols) continue;
        if (i > j) {
          const int t = i;
          i = j;
          j = t;
        }
        double* xi = X + (long long)i * nrows;
        double* xj = X + (long long)j * nrows;
        double a = 0.0, b = 0.0, g = 0.0;
        for (int r = threadIdx.x; r < nrows; r += kJacobiThreads) {
          const double u = xi[r], v = xj[r];
          a = fma(u, u, a);
          b = fma(v, v, b);
          g = fma(u, v, g);
        }
        block_sum3<kJacobiThreads>(a, b, g);
        if (!(a > 0.0) || !(b > 0.0)) continue;
        const double cosang = fabs(g) / (sqrt(a) * sqrt(b));
        if (a > tiny && b > tiny) local_max = fmax(local_max, cosang);
        if (!(cosang > tol)) continue;
        const double zeta = (b - a) / (2.0 * g);
        const double t = copysign(1.0, zeta) / (fabs(zeta) + hypot(1.0, zeta));
        const double c = 1.0 / sqrt(1.0 + t * t);
        const double sn = c * t;
        for (int r = threadIdx.x; r < nrows; r += kJacobiThreads) {
          const double u = xi[r], v = xj[r];
          xi[r] = c * u - sn * v;
          xj[r] = sn * u + c * v;
        }
        if (V) {
          double* vi = V + (long long)i * ncols;
          double* vj = V + (long long)j * ncols;
          for (int r = threadIdx.x; r < ncols; r += kJacobiThreads) {
            const double u = vi[r], v = vj[r];
            vi[r] = c * u - sn * v;
            vj[r] = sn * u + c * v;
          }
        }
        __syncthreads();
      }
      if (!grid_barrier(fl, nblocks)) return;
      // every block has read the previous sweep's slot before this barrier, so
      // the slot of the next sweep can be cleared now
      if (step == 0 && blockIdx.x == 0 && threadIdx.x == 0)
        atomicExch(&fl->off_max[(sweep + 1) & 1], 0ull);
    }
    if (threadIdx.x == 0 && local_max > 0.0)
      atomicMax(&fl->off_max[sweep & 1], (unsigned long long)__double_as_longlong(local_max));
    if (!grid_barrier(fl, nblocks)) return;
    const double m = __longlong_as_double(
        (long long)(*(volatile unsigned long long*)&fl->off_max[sweep & 1]));
    if (!(m > tol)) {  // converged (all blocks read the same value)
      if (blockIdx.x == 0 && threadIdx.x == 0) fl->sweeps = sweep + 1;
      return;
    }
  }
  if (blockIdx.x == 0 && threadIdx.x == 0) {
    fl->sweeps = max_sweeps;
    atomicExch(&fl->noconv, 1);
  }
}

// Values-only variant: one warp per column pair (eight pairs per block in
// flight), warp-shuffle reductions, so the FP64 latency of several pairs
// overlaps within a step.  Same rotation, ordering and stopping rule.
__global__ void __launch_bounds__(kJacobiThreads)
jacobi_warp_kernel(double* __restrict__ Xall, int nrows, int ncols, int npad, DevFlags* fl,
                   int max_sweeps, double tol, int nprob, long long pstride, double tiny_rel,
                   double* __restrict__ V) {
  const unsigned nblocks = gridDim.x;
  const int npairs = npad / 2;
  const int lane = threadIdx.x % 32;
  const int gwarp = blockIdx.x * (kJacobiThreads / 32) + threadIdx.x / 32;
  const int nwarps = gridDim.x * (kJacobiThreads / 32);
  {
    double part = 0.0, z1 = 0.0, z2 = 0.0;
    const long long per = (long long)nrows * ncols;
    for (int p = 0; p < nprob; ++p)
      for (long long e = blockIdx.x * (long long)kJacobiThreads + threadIdx.x; e < per;
           e += (long long)gridDim.x * kJacobiThreads)
        part = fma(Xall[p * pstride + e], Xall[p * pstride + e], part);
    block_sum3<kJacobiThreads>(part, z1, z2);
    if (threadIdx.x == 0 && part > 0.0) atomicAdd(&fl->fro2, part);
    if (!grid_barrier(fl, nblocks)) return;
  }
  const double tiny = tiny_rel * (*(volatile double*)&fl->fro2);
  for (int sweep = 0; sweep < max_sweeps; ++sweep) {
    double local_max = 0.0;
    for (int step = 0; step < npad - 1; ++step) {
      for (int kk = gwarp; kk < npairs * nprob; kk += nwarps) {
        const int k = kk % npairs;
        double* X = Xall + (long long)(kk / npairs) * pstride;
        int i = rr_col(k, step, npad);
        int j = rr_col(npad - 1 - k, step, npad);
        if (i >= ncols || j >= ncols) continue;
        double* xi = X + (long long)i * nrows;
        double* xj = X + (long long)j * nrows;
        double a = 0.0, b = 0.0, g = 0.0;
        for (int r = lane; r < nrows; r += 32) {
          const double u = xi[r], v = xj[r];
          a = fma(u, u, a);
          b = fma(v, v, b);
          g = fma(u, v, g);
        }
        for (int o = 16; o > 0; o >>= 1) {
          a += __shfl_xor_sync(0xffffffffu, a, o);
          b += __shfl_xor_sync(0xffffffffu, b, o);
          g += __shfl_xor_sync(0xffffffffu, g, o);
        }
        if (!(a > 0.0) || !(b > 0.0)) continue;
        const double cosang = fabs(g) / (sqrt(a) * sqrt(b));
        if (a > tiny && b > tiny) local_max = fmax(local_max, cosang);
        if (!(cosang > tol)) continue;
        const double zeta = (b - a) / (2.0 * g);
        const double t = copysign(1.0, zeta) / (fabs(zeta) + hypot(1.0, zeta));
        const double c = 1.0 / sqrt(1.0 + t * t);
        const double sn = c * t;
        for (int r = lane; r < nrows; r += 32) {
          const double u = xi[r], v = xj[r];
          xi[r] = c * u - sn * v;
          xj[r] = sn * u + c * v;
        }
        if (V) {  // one problem only when the rotations are accumulated
          double* vi = V + (long long)i * ncols;
          double* vj = V + (long long)j * ncols;
          for (int r = lane; r < ncols; r += 32) {
            const double u = vi[r], v = vj[r];
            vi[r] = c * u - sn * v;
            vj[r] = sn * u + c * v;
          }
        }
      }
      if (!grid_barrier(fl, nblocks)) return;
      if (step == 0 && blockIdx.x == 0 && threadIdx.x == 0)
        atomicExch(&fl->off_max[(sweep + 1) & 1], 0ull);
    }
    // block maximum of the warps' local maxima, then one atomic per block
    __shared__ double s_max[kJacobiThreads / 32];
    for (int o = 16; o > 0; o >>= 1) local_max = fmax(local_max, __shfl_xor_sync(0xffffffffu, local_max, o));
    if (lane == 0) s_max[threadIdx.x / 32] = local_max;
    __syncthreads();
    if (threadIdx.x == 0) {
      double m = 0.0;
      for (int w = 0; w < kJacobiThreads / 32; ++w) m = fmax(m, s_max[w]);
      if (m > 0.0)
        atomicMax(&fl->off_max[sweep & 1], (unsigned long long)__double_as_longlong(m));
    }
    if (!grid_barrier(fl, nblocks)) return;
    const double m = __longlong_as_double(
        (long long)(*(volatile unsigned long long*)&fl->off_max[sweep & 1]));
    if (!(m > tol)) {
      if (blockIdx.x == 0 && threadIdx.x == 0) fl->sweeps = sweep + 1;
      return;
    }
  }
  if (blockIdx.x == 0 && threadIdx.x == 0) {
    fl->sweeps = max_sweeps;
    atomicExch(&fl->noconv, 1);
  }
}

// Values-only Jacobi without a grid barrier per round-robin step: column c of
// problem p carries a step counter ver[p][c] (steps of all sweeps so far that
// touched it).  The pair (i, j) of global step g waits, lane by lane with an
// acquire load, until both counters read g (the previous step of each column is
// done), rotates, then releases both counters to g + 1.  Warp w takes the pairs
// w, w + nwarps, ... of every step, steps in order; all warps are resident (a
// cooperative launch), so the earliest unfinished pair always has its inputs and
// the waits end.  One grid barrier per sweep collects the largest off-diagonal
// cosine for the stopping rule; every wait gives up after kBarrierCycleLimit
// clocks, records the error and the kernel returns.
__device__ __forceinline__ int ld_acquire_s32(const int* p) {
  int v;
  asm volatile("ld.acquire.gpu.global.s32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
  return v;
}

__device__ __forceinline__ void st_release_s32(int* p, int v) {
  asm volatile("st.release.gpu.global.s32 [%0], %1;" ::"l"(p), "r"(v) : "memory");
}

// T = float: the same sweeps in FP32 with the rotations also applied to V
// (ncols x ncols column-major per problem, vstride apart), as a preconditioner
// for the FP64 run; its sweep cap is not an error (set_noconv = 0).
template <typename T>
__global__ void __launch_bounds__(kJacobiThreads)
jacobi_flow_kernel(T* __restrict__ Xall, int nrows, int ncols, int npad, DevFlags* fl,
                   int max_sweeps, double tol, int nprob, long long pstride, double tiny_rel,
                   int* __restrict__ ver, T* __restrict__ Vall, long long vstride, int set_noconv) {
  const unsigned nblocks = gridDim.x;
  const int npairs = npad / 2;
  const int lane = threadIdx.x % 32;
  const int gwarp = blockIdx.x * (kJacobiThreads / 32) + threadIdx.x / 32;
  const int nwarps = gridDim.x * (kJacobiThreads / 32);
  {
    double part = 0.0, z1 = 0.0, z2 = 0.0;
    const long long per = (long long)nrows * ncols;
    for (int p = 0; p < nprob; ++p)
      for (long long e = blockIdx.x * (long long)kJacobiThreads + threadIdx.x; e < per;
           e += (long long)gridDim.x * kJacobiThreads)
        part = fma((double)Xall[p * pstride + e], (double)Xall[p * pstride + e], part);
    block_sum3<kJacobiThreads>(part, z1, z2);
    if (threadIdx.x == 0 && part > 0.0) atomicAdd(&fl->fro2, part);
    if (!grid_barrier(fl, nblocks)) return;
  }
  const T tiny = (T)(tiny_rel * (*(volatile double*)&fl->fro2));
  const T ttol = (T)tol;
  bool failed = false;
  for (int sweep = 0; sweep < max_sweeps; ++sweep) {
    double local_max = 0.0;
    for (int step = 0; step < npad - 1 && !failed; ++step) {
      const int g = sweep * (npad - 1) + step;  // global step number
      for (int kk = gwarp; kk < npairs * nprob; kk += nwarps) {
        const int k = kk % npairs, p = kk / npairs;
        T* X = Xall + (long long)p * pstride;
        int* v = ver + (long long)p * npad;
        const int i = rr_col(k, step, npad);
        const int j = rr_col(npad - 1 - k, step, npad);
        // wait for both columns to have finished the previous step
        const long long t0 = clock64();
        while (ld_acquire_s32(v + i) < g || ld_acquire_s32(v + j) < g) {
          if (clock64() - t0 > kBarrierCycleLimit || *(volatile int*)&fl->error) {
            atomicExch(&fl->error, 1);
            failed = true;
            break;
          }
        }
        if (failed) break;
        if (i < ncols && j < ncols) {
          T* xi = X + (long long)i * nrows;
          T* xj = X + (long long)j * nrows;
          T a = 0, b = 0, gg = 0;
          for (int r = lane; r < nrows; r += 32) {
            const T u = xi[r], w = xj[r];
            a = fma(u, u, a);
            b = fma(w, w, b);
            gg = fma(u, w, gg);
          }
          for (int o = 16; o > 0; o >>= 1) {
            a += __shfl_xor_sync(0xffffffffu, a, o);
            b += __shfl_xor_sync(0xffffffffu, b, o);
            gg += __shfl_xor_sync(0xffffffffu, gg, o);
          }
          if (a > T(0) && b > T(0)) {
            const T cosang = fabs(gg) / (sqrt(a) * sqrt(b));
            if (a > tiny && b > tiny) local_max = fmax(local_max, (double)cosang);
            if (cosang > ttol) {
              const T zeta = (b - a) / (T(2) * gg);
              const T t = copysign(T(1), zeta) / (fabs(zeta) + hypot(T(1), zeta));
              const T c = T(1) / sqrt(T(1) + t * t);
              const T sn = c * t;
              for (int r = lane; r < nrows; r += 32) {
                const T u = xi[r], w = xj[r];
                xi[r] = c * u - sn * w;
                xj[r] = sn * u + c * w;
              }
              if (Vall) {
                T* vi = Vall + (long long)p * vstride + (long long)i * ncols;
                T* vj = Vall + (long long)p * vstride + (long long)j * ncols;
                for (int r = lane; r < ncols; r += 32) {
                  const T u = vi[r], w = vj[r];
                  vi[r] = c * u - sn * w;
                  vj[r] = sn * u + c * w;
                }
              }
            }
          }
        }
        __syncwarp();
        if (lane == 0) {
          __threadfence();
          st_release_s32(v + i, g + 1);
          st_release_s32(v + j, g + 1);
        }
        __syncwarp();
      }
    }
    __shared__ double s_max[kJacobiThreads / 32];
    for (int o = 16; o > 0; o >>= 1) local_max = fmax(local_max, __shfl_xor_sync(0xffffffffu, local_max, o));
    if (lane == 0) s_max[threadIdx.x / 32] = local_max;
    __syncthreads();
    if (threadIdx.x == 0) {
      double m = 0.0;
      for (int w = 0; w < kJacobiThreads / 32; ++w) m = fmax(m, s_max[w]);
      if (m > 0.0)
        atomicMax(&fl->off_max[sweep & 1], (unsigned long long)__double_as_longlong(m));
    }
    if (!grid_barrier(fl, nblocks)) return;
    const double m = __longlong_as_double(
        (long long)(*(volatile unsigned long long*)&fl->off_max[sweep & 1]));
    if (!(m > tol)) {
      if (blockIdx.x == 0 && threadIdx.x == 0) fl->sweeps = sweep + 1;
      return;
    }
    // every block has read this sweep's maximum: clear the slot of the next sweep
    if (blockIdx.x == 0 && threadIdx.x == 0) atomicExch(&fl->off_max[(sweep + 1) & 1], 0ull);
    if (!grid_barrier(fl, nblocks)) return;
  }
  if (blockIdx.x == 0 && threadIdx.x == 0) {
    fl->sweeps = max_sweeps;
    if (set_noconv) atomicExch(&fl->noconv, 1);
  }
}

__global__ void identity_kernel(double* x, int n) {
  const long long nn = (long long)n * n;
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < nn;
       i += (long long)gridDim.x * blockDim.x)
    x[i] = (i / n == i % n) ? 1.0 : 0.0;
}

cudaError_t fill_identity(cudaStream_t s, double* x, int n) {
  long long blocks = ((long long)n * n + 255) / 256;
  if (blocks > 4096) blocks = 4096;
  if (blocks < 1) blocks = 1;
  identity_kernel<<<(unsigned)blocks, 256, 0, s>>>(x, n);
  return cudaGetLastError();
}

int jacobi_batched(cudaStream_t s, double* X, int nrows, int ncols, int nprob, long long pstride,
                   DevFlags* flags, int max_sweeps, long long* launches, double tol_override,
                   bool serialize, int* colver);

// Cooperative launches rely on all their blocks being resident at once; two of
// them running together (different contexts or streams) could each hold SMs
// the other waits for.  They are therefore all issued on one stream per device,
// ordered after and before the caller's stream with events.
static std::mutex g_coop_mu;
static cudaStream_t g_coop[64] = {};

cudaStream_t coop_stream() {
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= 64) return nullptr;
  std::lock_guard<std::mutex> lock(g_coop_mu);
  if (!g_coop[dev] && cudaStreamCreateWithFlags(&g_coop[dev], cudaStreamNonBlocking) != cudaSuccess) {
    cudaGetLastError();
    g_coop[dev] = nullptr;
  }
  return g_coop[dev];
}

// Launch fn on the cooperative stream, ordered after the work so far on s and
// before the work issued later on s.
// An event record that becomes an event-record node when the stream is being
// captured into a CUDA graph (so that every replay records it).
static void record_event(cudaEvent_t ev, cudaStream_t s) {
  cudaStreamCaptureStatus st = cudaStreamCaptureStatusNone;
  if (cudaStreamIsCapturing(s, &st) == cudaSuccess && st == cudaStreamCaptureStatusActive)
    cudaEventRecordWithFlags(ev, s, cudaEventRecordExternal);
  else
    cudaEventRecord(ev, s);
}

static cudaError_t launch_coop_ordered(const void* fn, dim3 grid, dim3 block, void** args,
                                       cudaStream_t s, bool serialize, size_t smem = 0,
                                       cudaEvent_t t0 = nullptr, cudaEvent_t t1 = nullptr) {
  cudaStream_t cs = serialize ? coop_stream() : nullptr;
  if (!cs) {
    if (t0) record_event(t0, s);
    const cudaError_t r = cudaLaunchCooperativeKernel(fn, grid, block, args, smem, s);
    if (t1) record_event(t1, s);
    return r;
  }
  cudaEvent_t e1, e2;
  if (cudaEventCreateWithFlags(&e1, cudaEventDisableTiming) != cudaSuccess) return cudaErrorUnknown;
  if (cudaEventCreateWithFlags(&e2, cudaEventDisableTiming) != cudaSuccess) {
    cudaEventDestroy(e1);
    return cudaErrorUnknown;
  }
  cudaError_t e = cudaEventRecord(e1, s);
  if (e == cudaSuccess) e = cudaStreamWaitEvent(cs, e1, 0);
  // timing events on the cooperative stream bracket the kernel alone (that
  // stream runs one cooperative kernel at a time)
  if (e == cudaSuccess && t0) record_event(t0, cs);
  if (e == cudaSuccess) e = cudaLaunchCooperativeKernel(fn, grid, block, args, smem, cs);
  if (e == cudaSuccess && t1) record_event(t1, cs);
  if (e == cudaSuccess) e = cudaEventRecord(e2, cs);
  if (e == cudaSuccess) e = cudaStreamWaitEvent(s, e2, 0);
  cudaEventDestroy(e1);
  cudaEventDestroy(e2);
  return e;
}

cudaError_t launch_cooperative(const void* fn, dim3 grid, dim3 block, void** args, size_t smem,
                               cudaStream_t s, cudaEvent_t t0, cudaEvent_t t1) {
  return launch_coop_ordered(fn, grid, block, args, s, true, smem, t0, t1);
}

int jacobi_onesided(cudaStream_t s, double* X, int nrows, int ncols, double* V, DevFlags* flags,
                    int max_sweeps, long long* launches) {
  if (!V) return jacobi_batched(s, X, nrows, ncols, 1, 0, flags, max_sweeps, launches, 0.0, true);
  if (ncols < 2) {
    if (V && ncols == 1) {
      if (fill_identity(s, V, 1) != cudaSuccess) return -3;
      ++*launches;
    }
    return 0;
  }
  if (V) {
    if (fill_identity(s, V, ncols) != cudaSuccess) return -3;
    ++*launches;
  }
  const int npad = ncols + (ncols & 1);
  int dev = 0, nsm = 0, per_sm = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev);
  cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, jacobi_kernel, kJacobiThreads, 0);
  if (per_sm < 1) return -3;
  if (cudaMemsetAsync(flags, 0, kDevFlagsResetBytes, s) != cudaSuccess) return -3;
  const double tol = 2.220446049250313e-16 * std::sqrt((double)(nrows > 1 ? nrows : 1));
  int nprob = 1;
  long long pstride = 0;
  double tiny_rel = 1e-32;
  if (nrows <= kWarpJacobiMaxRows) {
    // one warp per column pair (eight per block): the FP64 latency of several
    // pairs overlaps; same rotation, ordering and stopping rule
    long long want = ((long long)(npad / 2) + kJacobiThreads / 32 - 1) / (kJacobiThreads / 32);
    const int wgrid = (int)(want < (long long)nsm ? want : (long long)nsm);
    void* wargs[] = {&X, &nrows, &ncols, (void*)&npad, &flags, &max_sweeps, (void*)&tol,
                     &nprob, &pstride, &tiny_rel, &V};
    if (launch_coop_ordered((void*)jacobi_warp_kernel, dim3(wgrid), dim3(kJacobiThreads), wargs,
                            s, true) != cudaSuccess)
      return -3;
    ++*launches;
    return 0;
  }
  int grid = npad / 2;
  if (grid > nsm) grid = nsm;  // one block per SM: fewer arrivals per barrier
  void* args[] = {&X, &nrows, &ncols, (void*)&npad, &V, &flags, &max_sweeps, (void*)&tol,
                  &nprob, &pstride, &tiny_rel};
  if (launch_coop_ordered((void*)jacobi_kernel, dim3(grid), dim3(kJacobiThreads), args, s, true) !=
      cudaSuccess)
    return -3;
  ++*launches;
  return 0;
}

// nprob independent problems X + p * pstride (same shape, no rotation
// accumulation) in one cooperative launch: one grid barrier per round-robin
// step serves all of them.
int jacobi_batched(cudaStream_t s, double* X, int nrows, int ncols, int nprob, long long pstride,
                   DevFlags* flags, int max_sweeps, long long* launches, double tol_override,
                   bool serialize, int* colver) {
  if (ncols < 2 || nprob < 1) return 0;
  const int npad = ncols + (ncols & 1);
  int dev = 0, nsm = 0, per_sm = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev);
  cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, jacobi_kernel, kJacobiThreads, 0);
  if (per_sm < 1) return -3;
  const bool warp_mode = tol_override > 0.0;  // values only: one warp per pair
  const long long per_block = warp_mode ? kJacobiThreads / 32 : 1;
  long long want = ((long long)(npad / 2) * nprob + per_block - 1) / per_block;
  int grid = (int)(want < (long long)nsm ? want : (long long)nsm);  // one block per SM
  if (cudaMemsetAsync(flags, 0, kDevFlagsResetBytes, s) != cudaSuccess) return -3;
  const double tol = tol_override > 0.0
                         ? tol_override
                         : 2.220446049250313e-16 * std::sqrt((double)(nrows > 1 ? nrows : 1));
  double* V = nullptr;
  double tiny_rel = warp_mode ? 1e-24 : 1e-32;
  if (warp_mode && colver) {  // step counters instead of a grid barrier per step
    if (cudaMemsetAsync(colver, 0, sizeof(int) * (size_t)nprob * npad, s) != cudaSuccess)
      return -3;
    double* Vnone = nullptr;
    long long vstride = 0;
    int set_noconv = 1;
    void* fargs[] = {&X, &nrows, &ncols, (void*)&npad, &flags, &max_sweeps, (void*)&tol,
                     &nprob, &pstride, &tiny_rel, &colver, &Vnone, &vstride, &set_noconv};
    if (launch_coop_ordered((void*)jacobi_flow_kernel<double>, dim3(grid), dim3(kJacobiThreads),
                            fargs, s, serialize) != cudaSuccess)
      return -3;
    ++*launches;
    return 0;
  }
  if (warp_mode) {
    void* wargs[] = {&X, &nrows, &ncols, (void*)&npad, &flags, &max_sweeps, (void*)&tol,
                     &nprob, &pstride, &tiny_rel, &V};
    if (launch_coop_ordered((void*)jacobi_warp_kernel, dim3(grid), dim3(kJacobiThreads), wargs, s,
                            serialize) != cudaSuccess)
      return -3;
    ++*launches;
    return 0;
  }
  void* args[] = {&X, &nrows, &ncols, (void*)&npad, &V, &flags, &max_sweeps, (void*)&tol,
                  &nprob, &pstride, &tiny_rel};
  if (launch_coop_ordered((void*)jacobi_kernel, dim3(grid), dim3(kJacobiThreads), args, s,
                          serialize) != cudaSuccess)
    return -3;
  ++*launches;
  return 0;
}

// ---------------------------------------------------------------------------
// Norms, sorting, gathering
// ---------------------------------------------------------------------------
__global__ void colnorm_kernel(const double* __restrict__ X, int nrows, int ncols,
                               double* __restrict__ sig) {
  const int warp = (blockIdx.x * blockDim.x + threadIdx.x) / 32;
  const int lane = threadIdx.x % 32;
  if (warp >= ncols) return;
  const double* x = X + (long long)warp * nrows;
  double acc = 0.0;
  for (int r = lane; r < nrows; r += 32) acc = fma(x[r], x[r], acc);
  for (int o = 16; o > 0; o >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, o);
  if (lane == 0) sig[warp] = sqrt(acc);
}

__global__ void rank_kernel(const double* __restrict__ sig, int n, int* __restrict__ perm) {
  for (int j = blockIdx.x * blockDim.x + threadIdx.x; j < n; j += gridDim.x * blockDim.x) {
    const double sj = sig[j];
    int rank = 0;
    for (int i = 0; i < n; ++i) {
      const double si = sig[i];
      rank += (si > sj) || (si == sj && i < j);
    }
    perm[rank] = j;
  }
}

cudaError_t column_norms_sorted(cudaStream_t s, const double* X, int nrows, int ncols, double* sig,
                                int* perm) {
  const int warps_per_block = 8;
  colnorm_kernel<<<(ncols + warps_per_block - 1) / warps_per_block, 32 * warps_per_block, 0, s>>>(
      X, nrows, ncols, sig);
  rank_kernel<<<(ncols + 255) / 256, 256, 0, s>>>(sig, ncols, perm);
  return cudaGetLastError();
}

__global__ void gather_cols_kernel(double* __restrict__ U, int rows, int k,
                                   const double* __restrict__ X, const double* __restrict__ V,
                                   const double* __restrict__ sig, const int* __restrict__ perm) {
  const int r = blockIdx.x;
  const int c = perm[r];
  __shared__ double best_v[256];
  __shared__ int best_i[256];
  const double inv = V ? 1.0 : (sig[c] > 0.0 ? 1.0 / sig[c] : 0.0);
  const double* src = V ? V + (long long)c * rows : X + (long long)c * rows;
  double bv = -1.0;
  int bi = 0x7fffffff;
  for (int i = threadIdx.x; i < rows; i += blockDim.x) {
    const double v = src[i] * inv;
    U[(long long)i * k + r] = v;
    if (fabs(v) > bv) {
      bv = fabs(v);
      bi = i;
    }
  }
  best_v[threadIdx.x] = bv;
  best_i[threadIdx.x] = bi;
  __syncthreads();
  for (int o = blockDim.x / 2; o > 0; o >>= 1) {
    if (threadIdx.x < o) {
      const double ov = best_v[threadIdx.x + o];
      const int oi = best_i[threadIdx.x + o];
      if (ov > best_v[threadIdx.x] || (ov == best_v[threadIdx.x] && oi < best_i[threadIdx.x])) {
        best_v[threadIdx.x] = ov;
        best_i[threadIdx.x] = oi;
      }
    }
    __syncthreads();
  }
  const int im = best_i[0];
  const bool flip = im < rows && U[(long long)im * k + r] < 0.0;
  __syncthreads();
  if (flip)
    for (int i = threadIdx.x; i < rows; i += blockDim.x) U[(long long)i * k + r] = -U[(long long)i * k + r];
}

cudaError_t gather_sorted_columns(cudaStream_t s, double* U, int rows, int k, const double* X,
                                  const double* V, const double* sig, const int* perm) {
  if (k <= 0) return cudaSuccess;
  gather_cols_kernel<<<k, 256, 0, s>>>(U, rows, k, X, V, sig, perm);
  return cudaGetLastError();
}

// ---------------------------------------------------------------------------
// Frobenius normalisation (deterministic two-level reduction)
// ---------------------------------------------------------------------------
constexpr int kNormBlocks = 304;

__global__ void sumsq_partial_kernel(const double* __restrict__ x, long long n,
                                     double* __restrict__ partial) {
  double acc = 0.0;
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n;
       i += (long long)gridDim.x * blockDim.x)
    acc = fma(x[i], x[i], acc);
  double b = 0.0, c = 0.0;
  block_sum3<256>(acc, b, c);
  if (threadIdx.x == 0) partial[blockIdx.x] = acc;
}

__global__ void scale_by_norm_kernel(double* __restrict__ x, long long n,
                                     const double* __restrict__ partial, int nparts,
                                     double* __restrict__ norm_out, int* __restrict__ bad) {
  __shared__ double s_norm;
  if (threadIdx.x == 0) {
    double t = 0.0;
    for (int i = 0; i < nparts; ++i) t += partial[i];
    s_norm = sqrt(t);
  }
  __syncthreads();
  const double nrm = s_norm;
  if (!(nrm > 0.0) || !isfinite(nrm)) {
    if (blockIdx.x == 0 && threadIdx.x == 0) atomicExch(bad, 1);
    return;
  }
  if (blockIdx.x == 0 && threadIdx.x == 0 && norm_out) *norm_out = nrm;
  const double inv = 1.0 / nrm;
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n;
       i += (long long)gridDim.x * blockDim.x)
    x[i] *= inv;
}

cudaError_t normalize_f64(cudaStream_t s, double* x, long long n, double* scratch, int* bad) {
  // scratch: kNormBlocks + 1 doubles (partials, then the norm)
  sumsq_partial_kernel<<<kNormBlocks, 256, 0, s>>>(x, n, scratch);
  scale_by_norm_kernel<<<kNormBlocks, 256, 0, s>>>(x, n, scratch, kNormBlocks,
                                                   scratch + kNormBlocks, bad);
  return cudaGetLastError();
}

// ---------------------------------------------------------------------------
// Blocked Cholesky pieces (CholeskyQR): a 32x32 diagonal block factorised by
// one CTA (pivots floored at `floor`, counted in *floored), its triangular
// inverse, Gram scaling by the column norms with an optional diagonal shift
// (shifted CholeskyQR: Fukaya, Kannan, Nakatsukasa, Yamamoto & Yanagisawa,
// SIAM J. Sci. Comput. 42, A477 (2020)), and a strided copy.
// ---------------------------------------------------------------------------
// One block of 128 threads (all four schedulers of the SM, whose FP64 pipes are
// narrow): right-looking Cholesky of the (<= 32 x 32) diagonal block in shared
// memory -- one thread takes the pivot, the column scaling and the rank-1
// update of the trailing triangle are spread over the block -- then the
// inverse row by row, x_i = (e_i - sum_k L_ik x_k) / L_ii, with the sum over k
// split into four partial sums per column.
constexpr int kCholThreads = 128;

__global__ void __launch_bounds__(kCholThreads)
chol_diag_kernel(double* __restrict__ G, int lda, int j0, int jb, double* __restrict__ Linv,
                 double floor, int* floored, double tau, int* __restrict__ defmask) {
  __shared__ double L[32][33];
  __shared__ double X[32][33];
  __shared__ double rinv[32];
  __shared__ double part[4][32];
  __shared__ int s_def;
  const int t = threadIdx.x;
  for (int e = t; e < 32 * 32; e += kCholThreads) {
    const int i = e / 32, j = e % 32;
    L[i][j] = (i < jb && j < jb && j <= i) ? G[(long long)(j0 + i) * lda + j0 + j] : 0.0;
  }
  __syncthreads();
  for (int k = 0; k < jb; ++k) {
    if (t == 0) {
      double dkk = L[k][k];
      s_def = 0;
      if (defmask && !(dkk > tau)) {  // column k lies in the span of the earlier ones
        s_def = 1;
        defmask[j0 + k] = 1;
        dkk = 1.0;
      } else if (!(dkk > floor)) {
        dkk = floor;
        atomicAdd(floored, 1);
      }
      const double piv = sqrt(dkk);
      L[k][k] = piv;
      rinv[k] = 1.0 / piv;
    }
    __syncthreads();
    const int m = jb - k - 1;  // rows below the pivot
    if (t < m) L[k + 1 + t][k] = s_def ? 0.0 : L[k + 1 + t][k] * rinv[k];
    __syncthreads();
    // trailing triangle: (i, j) with k < j <= i < jb
    for (int e = t; e < m * m; e += kCholThreads) {
      const int i = k + 1 + e / m, j = k + 1 + e % m;
      if (j <= i) L[i][j] -= L[i][k] * L[j][k];
    }
    __syncthreads();
  }
  for (int e = t; e < jb * jb; e += kCholThreads) {
    const int i = e / jb, j = e % jb;
    G[(long long)(j0 + i) * lda + j0 + j] = (j <= i) ? L[i][j] : 0.0;
  }
  // inverse: thread t handles column j = t % 32 and quarter q = t / 32 of the k range
  const int jc = t % 32, q = t / 32;
  for (int i = 0; i < 32; ++i) {
    double acc = 0.0;
    for (int k = q; k < i; k += 4) acc -= L[i][k] * X[k][jc];
    part[q][jc] = acc;
    __syncthreads();
    if (q == 0)
      X[i][jc] = (i < jb && jc <= i)
                     ? ((i == jc ? 1.0 : 0.0) + part[0][jc] + part[1][jc] + part[2][jc] +
                        part[3][jc]) * rinv[i]
                     : 0.0;
    __syncthreads();
  }
  for (int e = t; e < 32 * 32; e += kCholThreads) {
    const int i = e / 32, j = e % 32;
    Linv[i * 32 + j] = (i < jb && j < jb) ? X[i][j] : 0.0;
  }
}

cudaError_t chol_diag(cudaStream_t s, double* G, int lda, int j0, int jb, double* Linv,
                      double floor, int* floored, double tau, int* defmask) {
  chol_diag_kernel<<<1, kCholThreads, 0, s>>>(G, lda, j0, jb, Linv, floor, floored, tau, defmask);
  return cudaGetLastError();
}

// Replace every column j of Q (row-major rows x n) with defmask[j] set by
// Gaussian values, then clear the mask.  One block per column.
__device__ __forceinline__ unsigned long long splitmix64(unsigned long long z);

__global__ void replace_flagged_kernel(double* __restrict__ Q, int rows, int n,
                                       int* __restrict__ defmask, unsigned long long seed) {
  const int j = blockIdx.x;
  if (!defmask[j]) return;
  for (int i = threadIdx.x; i < rows; i += blockDim.x) {
    const unsigned long long base =
        seed * 0xD1B54A32D192ED03ull + 2ull * ((unsigned long long)j * rows + i);
    const unsigned long long z1 = splitmix64(base), z2 = splitmix64(base + 1ull);
    const double u1 = ((double)(z1 >> 11) + 1.0) * 0x1.0p-53;
    const double u2 = (double)(z2 >> 11) * 0x1.0p-53;
    Q[(long long)i * n + j] = sqrt(-2.0 * log(u1)) * cospi(2.0 * u2);
  }
  __syncthreads();
  if (threadIdx.x == 0) defmask[j] = 0;
}

cudaError_t replace_flagged(cudaStream_t s, double* Q, int rows, int n, int* defmask,
                            unsigned long long seed) {
  replace_flagged_kernel<<<n, 256, 0, s>>>(Q, rows, n, defmask, seed);
  return cudaGetLastError();
}

// d[i] = sqrt(G[i][i]) (or 1 if zero), then G[i][j] /= d[i] d[j] and
// G[i][i] += shift_rel * n (the trace of the scaled Gram is n).
__global__ void gram_diag_kernel(const double* __restrict__ G, int n, double* __restrict__ d) {
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
    const double g = G[(long long)i * n + i];
    d[i] = g > 0.0 ? sqrt(g) : 1.0;
  }
}

__global__ void gram_scale_kernel(double* __restrict__ G, int n, const double* __restrict__ d,
                                  double shift) {
  const long long nn = (long long)n * n;
  for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < nn;
       e += (long long)gridDim.x * blockDim.x) {
    const long long i = e / n, j = e - i * n;
    double v = G[e] / (d[i] * d[j]);
    if (i == j) v += shift;
    G[e] = v;
  }
}

cudaError_t gram_scale(cudaStream_t s, double* G, int n, double* d, double shift_rel) {
  gram_diag_kernel<<<(n + 255) / 256, 256, 0, s>>>(G, n, d);
  long long blocks = ((long long)n * n + 255) / 256;
  if (blocks > 1024) blocks = 1024;
  gram_scale_kernel<<<(unsigned)blocks, 256, 0, s>>>(G, n, d, shift_rel * n);
  return cudaGetLastError();
}

// dst[r * dld + c] = src[r * sld + c] * (colscale ? 1 / colscale[c0 + c] : 1), r < rows, c < cols
__global__ void copy2d_kernel(double* __restrict__ dst, long long dld, const double* __restrict__ src,
                              long long sld, int rows, int cols, const double* __restrict__ colscale,
                              int c0) {
  const long long n = (long long)rows * cols;
  for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < n;
       e += (long long)gridDim.x * blockDim.x) {
    const long long r = e / cols, c = e % cols;
    double v = src[r * sld + c];
    if (colscale) v /= colscale[c0 + c];
    dst[r * dld + c] = v;
  }
}

cudaError_t copy2d(cudaStream_t s, double* dst, long long dld, const double* src, long long sld,
                   int rows, int cols, const double* colscale, int c0) {
  long long blocks = ((long long)rows * cols + 255) / 256;
  if (blocks > 2048) blocks = 2048;
  if (blocks < 1) blocks = 1;
  copy2d_kernel<<<(unsigned)blocks, 256, 0, s>>>(dst, dld, src, sld, rows, cols, colscale, c0);
  return cudaGetLastError();
}

__global__ void count_nonfinite_kernel(const double* __restrict__ x, long long n, int* out) {
  int bad = 0;
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n;
       i += (long long)gridDim.x * blockDim.x)
    bad += !isfinite(x[i]);
  if (bad) atomicAdd(out, bad);
}

cudaError_t count_nonfinite(cudaStream_t s, const double* x, long long n, int* out) {
  long long blocks = (n + 255) / 256;
  if (blocks > 1024) blocks = 1024;
  if (blocks < 1) blocks = 1;
  count_nonfinite_kernel<<<(unsigned)blocks, 256, 0, s>>>(x, n, out);
  return cudaGetLastError();
}

// ---------------------------------------------------------------------------
// Counter-based Gaussian fill
// ---------------------------------------------------------------------------
__device__ __forceinline__ unsigned long long splitmix64(unsigned long long z) {
  z += 0x9E3779B97F4A7C15ull;
  z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
  z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
  return z ^ (z >> 31);
}

__global__ void gaussian_kernel(double* __restrict__ x, long long n, unsigned long long seed) {
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n;
       i += (long long)gridDim.x * blockDim.x) {
    const unsigned long long base = seed * 0xD1B54A32D192ED03ull + 2ull * (unsigned long long)i;
    const unsigned long long z1 = splitmix64(base), z2 = splitmix64(base + 1ull);
    const double u1 = ((double)(z1 >> 11) + 1.0) * 0x1.0p-53;  // (0, 1]
    const double u2 = (double)(z2 >> 11) * 0x1.0p-53;          // [0, 1)
    x[i] = sqrt(-2.0 * log(u1)) * cospi(2.0 * u2);
  }
}

cudaError_t gaussian_fill(cudaStream_t s, double* x, long long n, unsigned long long seed) {
  long long blocks = (n + 255) / 256;
  if (blocks > 4096) blocks = 4096;
  if (blocks < 1) blocks = 1;
  gaussian_kernel<<<(unsigned)blocks, 256, 0, s>>>(x, n, seed);
  return cudaGetLastError();
}


// ---------------------------------------------------------------------------
// FP32 preconditioning of the values-only Jacobi (corner spectra)
// ---------------------------------------------------------------------------
// X (column-major n1 x n2, FP32) = C (row-major n1 x n2, FP64), V = identity.
__global__ void corner_f32_kernel(const double* __restrict__ C, float* __restrict__ X,
                                  float* __restrict__ V, int n1, int n2) {
  const long long nn = (long long)n1 * n2, vv = (long long)n2 * n2;
  for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < nn + vv;
       e += (long long)gridDim.x * blockDim.x) {
    if (e < nn) {
      const long long i = e / n2, j = e % n2;  // reads along C's rows
      X[j * n1 + i] = (float)C[e];
    } else {
      const long long f = e - nn;
      V[f] = (f / n2 == f % n2) ? 1.f : 0.f;
    }
  }
}

// out (row-major n x n, FP64) = V (column-major n x n, FP32).
__global__ void v_f64_kernel(const float* __restrict__ V, double* __restrict__ out, int n) {
  const long long nn = (long long)n * n;
  for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < nn;
       e += (long long)gridDim.x * blockDim.x) {
    const long long i = e / n, j = e % n;
    out[e] = (double)V[j * n + i];
  }
}

int jacobi_precondition_f32(cudaStream_t s, const double* const* C, int n1, int n2, int nprob,
                            float* X, float* V, double* const* Vout, DevFlags* flags,
                            int max_sweeps, double tol, double tiny_rel, int* colver,
                            long long* launches) {
  if (n2 < 2 || nprob < 1 || n2 > n1) return -1;
  const long long pstride = (long long)n1 * n2, vstride = (long long)n2 * n2;
  for (int p = 0; p < nprob; ++p) {
    long long blocks = (pstride + vstride + 255) / 256;
    if (blocks > 4096) blocks = 4096;
    corner_f32_kernel<<<(unsigned)blocks, 256, 0, s>>>(C[p], X + p * pstride, V + p * vstride, n1,
                                                      n2);
    if (cudaGetLastError() != cudaSuccess) return -3;
    ++*launches;
  }
  const int npad = n2 + (n2 & 1);
  int dev = 0, nsm = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev);
  const long long want = ((long long)(npad / 2) * nprob + kJacobiThreads / 32 - 1) / (kJacobiThreads / 32);
  int grid = (int)(want < (long long)nsm ? want : (long long)nsm);
  if (cudaMemsetAsync(flags, 0, kDevFlagsResetBytes, s) != cudaSuccess ||
      cudaMemsetAsync(colver, 0, sizeof(int) * (size_t)nprob * npad, s) != cudaSuccess)
    return -3;
  int set_noconv = 0;
  void* fargs[] = {&X, &n1, &n2, (void*)&npad, &flags, &max_sweeps, (void*)&tol, &nprob,
                   (void*)&pstride, &tiny_rel, &colver, &V, (void*)&vstride, &set_noconv};
  if (launch_coop_ordered((void*)jacobi_flow_kernel<float>, dim3(grid), dim3(kJacobiThreads),
                          fargs, s, true) != cudaSuccess)
    return -3;
  ++*launches;
  for (int p = 0; p < nprob; ++p) {
    long long blocks = (vstride + 255) / 256;
    if (blocks > 4096) blocks = 4096;
    v_f64_kernel<<<(unsigned)blocks, 256, 0, s>>>(V + p * vstride, Vout[p], n2);
    if (cudaGetLastError() != cudaSuccess) return -3;
    ++*launches;
  }
  return 0;
}

}  // namespace ctm
