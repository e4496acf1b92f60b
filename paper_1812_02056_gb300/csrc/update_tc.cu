// tcgen05 tensor-core rank-s update (placeholder until the kernel lands).
#include "gb_internal.cuh"

namespace gb {
size_t tc_pack_bytes(int64_t M, int64_t N, int64_t K, bool nn) {
  (void)M; (void)N; (void)K; (void)nn;
  return 0;
}
cudaError_t launch_update_tc(const TcUpdateArgs &a, cudaStream_t st) {
  (void)a; (void)st;
  return cudaErrorNotSupported;
}
bool tc_supported(int device) { (void)device; return false; }
}  // namespace gb
