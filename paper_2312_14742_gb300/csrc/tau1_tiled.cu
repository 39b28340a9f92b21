// Tiled Tau1 step kernel (placeholder until the tiled kernel lands).
#include "kernels.h"

namespace lbm {

bool tau1_tiled_supported(int, int) { return false; }

cudaError_t launch_tau1_tiled(int, int, const StepArgs&, cudaStream_t) { return cudaErrorNotSupported; }

}  // namespace lbm
