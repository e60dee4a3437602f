// xpass_tc.cu -- tcgen05 tensor-core X pass for bfloat16 X (not yet enabled).
#include "internal.h"

namespace nmf {

bool xpass_tc_available() { return false; }
XPassPlan xpass_tc_plan(int n, int m, int nu, int num_sms) { return xpass_simt_plan(n, m, nu, num_sms); }
cudaError_t xpass_tc_launch(const XPassPlan& plan, const XPassArgs& a, cudaStream_t s) {
  return xpass_simt_launch(plan, a, true, s);
}

}  // namespace nmf
