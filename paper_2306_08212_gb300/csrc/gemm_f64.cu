// FP64 contraction kernel: a register-tiled GEMM whose operands are addressed
// through LegMaps, so a tensor contraction with any leg order runs without a
// separate transpose pass.  FP64 throughput on GB300 is low (a few FMA per
// clock per SM), so the kernel is arithmetic-bound for every shape used here;
// the gathers cost L2 traffic only.
#include "ctm_internal.h"

namespace ctm {

__device__ __forceinline__ long long map_offset(const LegMap& m, long long idx) {
  long long off = 0;
  for (int l = m.n - 1; l >= 0; --l) {
    const long long d = m.dim[l];
    const long long q = idx / d;
    off += (idx - q * d) * m.stride[l];
    idx = q;
  }
  return off;
}

template <int BM, int BN, int BK, int TM, int TN>
__global__ void __launch_bounds__((BM / TM) * (BN / TN))
gemm_f64_kernel(long long M, long long N, long long K, double alpha, const double* __restrict__ A,
                LegMap Am, LegMap Ak, const double* __restrict__ B, LegMap Bk, LegMap Bn,
                double beta, double* __restrict__ C, LegMap Cm, LegMap Cn, int a_m_fast,
                int b_n_fast, long long kchunk, double* __restrict__ partial) {
  constexpr int NT = (BM / TM) * (BN / TN);
  __shared__ double As[BK][BM + 1];
  __shared__ double Bs[BK][BN + 1];
  __shared__ long long offAm[BM], offCm[BM], offBn[BN], offCn[BN], offAk[BK], offBk[BK];

  const int tid = threadIdx.x;
  const long long m0 = (long long)blockIdx.y * BM;
  const long long n0 = (long long)blockIdx.x * BN;

  for (int i = tid; i < BM; i += NT) {
    const long long m = m0 + i;
    offAm[i] = m < M ? map_offset(Am, m) : 0;
    offCm[i] = m < M ? map_offset(Cm, m) : 0;
  }
  for (int j = tid; j < BN; j += NT) {
    const long long n = n0 + j;
    offBn[j] = n < N ? map_offset(Bn, n) : 0;
    offCn[j] = n < N ? map_offset(Cn, n) : 0;
  }

  const int tx = tid % (BN / TN);
  const int ty = tid / (BN / TN);
  double acc[TM][TN];
#pragma unroll
  for (int i = 0; i < TM; ++i)
#pragma unroll
    for (int j = 0; j < TN; ++j) acc[i][j] = 0.0;

  const long long kbeg = (long long)blockIdx.z * kchunk;
  const long long kend = kbeg + kchunk < K ? kbeg + kchunk : K;
  for (long long k0 = kbeg; k0 < kend; k0 += BK) {
    __syncthreads();
    for (int i = tid; i < BK; i += NT) {
      const long long k = k0 + i;
      offAk[i] = k < kend ? map_offset(Ak, k) : 0;
      offBk[i] = k < kend ? map_offset(Bk, k) : 0;
    }
    __syncthreads();
    for (int t = tid; t < BM * BK; t += NT) {
      const int mm = a_m_fast ? t % BM : t / BK;
      const int kk = a_m_fast ? t / BM : t % BK;
      const bool ok = (m0 + mm < M) && (k0 + kk < kend);
      As[kk][mm] = ok ? A[offAm[mm] + offAk[kk]] : 0.0;
    }
    for (int t = tid; t < BN * BK; t += NT) {
      const int nn = b_n_fast ? t % BN : t / BK;
      const int kk = b_n_fast ? t / BN : t % BK;
      const bool ok = (n0 + nn < N) && (k0 + kk < kend);
      Bs[kk][nn] = ok ? B[offBk[kk] + offBn[nn]] : 0.0;
    }
    __syncthreads();
#pragma unroll
    for (int kk = 0; kk < BK; ++kk) {
      double a[TM], b[TN];
#pragma unroll
      for (int i = 0; i < TM; ++i) a[i] = As[kk][ty * TM + i];
#pragma unroll
      for (int j = 0; j < TN; ++j) b[j] = Bs[kk][tx * TN + j];
#pragma unroll
      for (int i = 0; i < TM; ++i)
#pragma unroll
        for (int j = 0; j < TN; ++j) acc[i][j] = fma(a[i], b[j], acc[i][j]);
    }
  }
#pragma unroll
  for (int i = 0; i < TM; ++i) {
    const int mm = ty * TM + i;
    if (m0 + mm >= M) continue;
#pragma unroll
    for (int j = 0; j < TN; ++j) {
      const int nn = tx * TN + j;
      if (n0 + nn >= N) continue;
      const double v = alpha * acc[i][j];
      if (partial) {  // split-K: dense partial tile, reduced in a fixed order later
        partial[((long long)blockIdx.z * M + m0 + mm) * N + n0 + nn] = v;
        continue;
      }
      double* c = C + offCm[mm] + offCn[nn];
      *c = (beta == 0.0) ? v : fma(beta, *c, v);
    }
  }
}

static int innermost_unit(const LegMap& m) { return m.n > 0 && m.stride[m.n - 1] == 1; }

__global__ void splitk_reduce_kernel(const double* __restrict__ partial, int splits, long long M,
                                     long long N, double beta, double* __restrict__ C, LegMap Cm,
                                     LegMap Cn) {
  const long long MN = M * N;
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < MN;
       i += (long long)gridDim.x * blockDim.x) {
    double v = 0.0;
    for (int z = 0; z < splits; ++z) v += partial[z * MN + i];
    const long long m = i / N, n = i - m * N;
    double* c = C + map_offset(Cm, m) + map_offset(Cn, n);
    *c = (beta == 0.0) ? v : fma(beta, *c, v);
  }
}

cudaError_t gemm_f64(cudaStream_t s, long long M, long long N, long long K, double alpha,
                     const double* A, const LegMap& Am, const LegMap& Ak, const double* B,
                     const LegMap& Bk, const LegMap& Bn, double beta, double* C,
                     const LegMap& Cm, const LegMap& Cn) {
  if (M <= 0 || N <= 0) return cudaSuccess;
  const int a_m_fast = innermost_unit(Am) && !innermost_unit(Ak);
  const int b_n_fast = innermost_unit(Bn);
  const long long tiles64 = ((M + 63) / 64) * ((N + 63) / 64);
  if (tiles64 >= 2 * 152) {
    dim3 grid((unsigned)((N + 63) / 64), (unsigned)((M + 63) / 64));
    if (grid.y > 65535) return cudaErrorInvalidConfiguration;
    gemm_f64_kernel<64, 64, 16, 4, 4><<<grid, 256, 0, s>>>(M, N, K, alpha, A, Am, Ak, B, Bk, Bn,
                                                           beta, C, Cm, Cn, a_m_fast, b_n_fast, K,
                                                           nullptr);
    return cudaGetLastError();
  }
  const long long tiles32 = ((M + 31) / 32) * ((N + 31) / 32);
  if (tiles32 < 152 && K < 512) {
    // few output tiles and a short K: 16 x 16 tiles put more blocks on the SMs
    dim3 grid((unsigned)((N + 15) / 16), (unsigned)((M + 15) / 16));
    if (grid.y > 65535) return cudaErrorInvalidConfiguration;
    gemm_f64_kernel<16, 16, 16, 1, 1><<<grid, 256, 0, s>>>(M, N, K, alpha, A, Am, Ak, B, Bk, Bn,
                                                           beta, C, Cm, Cn, a_m_fast, b_n_fast, K,
                                                           nullptr);
    return cudaGetLastError();
  }
  // few output tiles and a long K: split K over more blocks, reduce deterministically
  long long splits = 1;
  if (tiles32 < 2 * 152 && K >= 512) {
    splits = (2 * 152 + tiles32 - 1) / tiles32;
    const long long kmax = K / 256;
    if (splits > kmax) splits = kmax;
    if (splits > 64) splits = 64;
    if (splits < 1) splits = 1;
  }
  const long long kchunk = ((K + splits - 1) / splits + 15) / 16 * 16;
  splits = (K + kchunk - 1) / kchunk;
  dim3 grid((unsigned)((N + 31) / 32), (unsigned)((M + 31) / 32), (unsigned)splits);
  if (grid.y > 65535) return cudaErrorInvalidConfiguration;
  double* partial = nullptr;
  if (splits > 1) {
    cudaError_t e = cudaMallocAsync(&partial, sizeof(double) * splits * M * N, s);
    if (e != cudaSuccess) return e;
  }
  gemm_f64_kernel<32, 32, 16, 2, 2><<<grid, 256, 0, s>>>(M, N, K, alpha, A, Am, Ak, B, Bk, Bn,
                                                         beta, C, Cm, Cn, a_m_fast, b_n_fast,
                                                         kchunk, partial);
  if (splits > 1) {
    long long blocks = (M * N + 255) / 256;
    if (blocks > 4096) blocks = 4096;
    splitk_reduce_kernel<<<(unsigned)blocks, 256, 0, s>>>(partial, (int)splits, M, N, beta, C,
                                                          Cm, Cn);
    cudaFreeAsync(partial, s);
  }
  return cudaGetLastError();
}

__global__ void permute_f64_kernel(double* __restrict__ out, const double* __restrict__ in,
                                   LegMap map, long long n) {
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n;
       i += (long long)gridDim.x * blockDim.x)
    out[i] = in[map_offset(map, i)];
}

cudaError_t permute_f64(cudaStream_t s, double* out, const double* in, const LegMap& map) {
  const long long n = map.extent();
  if (n <= 0) return cudaSuccess;
  long long blocks = (n + 255) / 256;
  if (blocks > 152 * 16) blocks = 152 * 16;
  permute_f64_kernel<<<(unsigned)blocks, 256, 0, s>>>(out, in, map, n);
  return cudaGetLastError();
}

}  // namespace ctm
