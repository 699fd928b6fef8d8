// step_hub_bf16.cu -- long-row kernels (the neighbour lists of high-degree rows
// summed in segments by separate lane groups, then combined in segment order)
// with __nv_bfloat16 replica storage, one per (lanes per row G, 16-byte vectors per lane
// VPL) of the direct-gather kernels; the factory maps a shape to its kernel
// (nullptr if not built).
#include "step_impl.cuh"

namespace qqa {

using StepFn = void (*)(const InstDesc *, const Tile *, const int32_t *, RunStatus *, int32_t);

StepFn step_hub_kernel_bf16(int G, int VPL)
{
#define QQA_CASE(g, v) \
    if (G == g && VPL == v) return qqa_step_hub_kernel<__nv_bfloat16, g, v>;
    QQA_CASE(1, 1) QQA_CASE(1, 2) QQA_CASE(1, 4)
    QQA_CASE(2, 1) QQA_CASE(2, 2) QQA_CASE(2, 4)
    QQA_CASE(4, 1) QQA_CASE(4, 2) QQA_CASE(4, 4)
    QQA_CASE(8, 1) QQA_CASE(8, 2) QQA_CASE(8, 4)
    QQA_CASE(16, 1) QQA_CASE(16, 2) QQA_CASE(16, 4)
    QQA_CASE(32, 1) QQA_CASE(32, 2) QQA_CASE(32, 4)
#undef QQA_CASE
    return nullptr;
}

}  // namespace qqa
