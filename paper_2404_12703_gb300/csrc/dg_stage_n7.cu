// dg_stage_n7.cu -- the stage kernels of degree N = 7 in both precisions
// (FP64 and FP32-bulk) and all their launch variants; one translation unit
// per degree keeps the build parallel.
#include "dg_stage.cuh"

namespace dg {
DG_STAGE_ENTRY_POINTS(7)
}  // namespace dg
