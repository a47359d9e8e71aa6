// Kernels specific to the FP32-inner / FP64-refinement mode (filled in with that mode).
#include "common.cuh"
#include "launch.h"

namespace podcg {}  // namespace podcg
