// dg_stage_n1.cu -- the stage kernels of degree N = 1 in both precisions
// (FP64 and FP32-bulk) and all their launch variants; one translation unit
// per degree keeps the build parallel.
#include "dg_stage.cuh"

namespace dg {
DG_STAGE_ENTRY_POINTS(1)
}  // namespace dg
