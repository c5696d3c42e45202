// Precision-form kernels for fp16 storage (see h2_mixed_launch.cuh).
#include "h2_mixed_launch.cuh"

namespace h2i {
template h2_status mixed_pass_form<h2::kFormFp16>(const MixedLaunch&, unsigned, cudaStream_t, const TcPass*);
}  // namespace h2i
