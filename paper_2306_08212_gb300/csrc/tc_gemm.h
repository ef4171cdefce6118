// Tensor-core (tcgen05) contraction path for the TF32 / BF16 modes.
#pragma once
#include "ctm_internal.h"

namespace ctm {

struct TcGemm;

// Returns nullptr when the tensor-core path cannot be set up.
TcGemm* tc_create();
void tc_destroy(TcGemm* t);

// C(m, n) = sum_k A(m, k) B(k, n) with FP64 operands addressed through LegMaps
// and an FP64 result, computed with TF32 (precision 1) or BF16 (precision 2)
// products and FP32 accumulation.  A timed-out wait inside the kernel sets
// *err_word (device, or the object's own word when null).  When ev_begin/ev_end
// are given they are recorded around the GEMM kernel alone.  Returns 0 on success.
int tc_contract(TcGemm* t, cudaStream_t s, int precision, long long M, long long N, long long K,
                const double* A, const LegMap& Am, const LegMap& Ak, const double* B,
                const LegMap& Bk, const LegMap& Bn, double* C, const LegMap& Cm,
                const LegMap& Cn, long long* launches, int* err_word, cudaEvent_t ev_begin,
                cudaEvent_t ev_end);

// Device error word of t (1 after a timed-out wait); synchronises s.
int tc_error(TcGemm* t, cudaStream_t s);

}  // namespace ctm
