// The single-launch evaluator, wide tile form (int64 entries, leaves up to
// 32 rows), and the entry points for both forms (persist.cuh).
#include "persist.cuh"

cudaError_t persist_warps(int W, bool narrow, int sms, int64_t* warps) {
  return narrow ? persist_warps_narrow(W, sms, warps) : persist_warps_t<false>(W, sms, warps);
}

cudaError_t launch_persist(const PersistArgs& a, int W, bool narrow, int sms, cudaStream_t s) {
  return narrow ? launch_persist_narrow(a, W, sms, s) : launch_persist_t<false>(a, W, sms, s);
}
