// Precision-form kernels for int16 storage (see h2_mixed_launch.cuh).
#include "h2_mixed_launch.cuh"

namespace h2i {
template h2_status mixed_pass_form<h2::kFormInt16>(const MixedLaunch&, unsigned, cudaStream_t, const TcPass*);
}  // namespace h2i
