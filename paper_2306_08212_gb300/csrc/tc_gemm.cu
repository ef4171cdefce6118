// Placeholder until the tcgen05 kernels land: the mixed-precision modes report
// CTM_ERR_UNSUPPORTED instead of silently running in FP64.
#include "tc_gemm.h"

namespace ctm {

struct TcGemm {
  int unused;
};

TcGemm* tc_create() { return nullptr; }
void tc_destroy(TcGemm* t) { delete t; }

int tc_contract(TcGemm*, cudaStream_t, int, long long, long long, long long, const double*,
                const LegMap&, const LegMap&, const double*, const LegMap&, const LegMap&, double*,
                const LegMap&, const LegMap&, long long*) {
  return -6;
}

}  // namespace ctm
