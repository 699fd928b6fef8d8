// step_tiled_fp32.cu -- TMA-staged step kernels with float replica storage, one per
// (lanes per row G, vectors per lane VPL, row groups per warp RPW); the factory
// maps a shape to its kernel (nullptr if not built).
#include "step_impl.cuh"

namespace qqa {

using TiledFn = void (*)(const InstDesc *, const Tile *, const int32_t *, RunStatus *, int32_t, int32_t, int32_t);

TiledFn step_tiled_kernel_fp32(int G, int VPL, int RPW)
{
#define QQA_CASE(g, v, r) \
    if (G == g && VPL == v && RPW == r) return qqa_step_tiled_kernel<float, g, v, r>;
    QQA_CASE(4, 1, 2) QQA_CASE(4, 1, 4)
    QQA_CASE(8, 1, 2) QQA_CASE(8, 1, 4) QQA_CASE(8, 1, 8)
    QQA_CASE(16, 1, 2) QQA_CASE(16, 1, 4) QQA_CASE(16, 1, 8)
    QQA_CASE(32, 1, 2) QQA_CASE(32, 1, 4) QQA_CASE(32, 1, 8)
    QQA_CASE(32, 2, 2) QQA_CASE(32, 2, 4)
    QQA_CASE(32, 4, 2)
#undef QQA_CASE
    return nullptr;
}

}  // namespace qqa
