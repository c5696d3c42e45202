// Precision-form kernels for bf16 storage (see h2_mixed_launch.cuh).
#include "h2_mixed_launch.cuh"

namespace h2i {
template h2_status mixed_pass_form<h2::kFormBf16>(const MixedLaunch&, unsigned, cudaStream_t, const TcPass*);
}  // namespace h2i
