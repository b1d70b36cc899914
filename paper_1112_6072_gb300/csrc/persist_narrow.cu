// The single-launch evaluator, narrow tile form (int32 entries, leaves up to
// 16 rows), compiled apart from the wide form (persist.cuh).
#include "persist.cuh"

cudaError_t persist_warps_narrow(int W, int sms, int64_t* warps) { return persist_warps_t<true>(W, sms, warps); }

cudaError_t launch_persist_narrow(const PersistArgs& a, int W, int sms, cudaStream_t s) {
  return launch_persist_t<true>(a, W, sms, s);
}
