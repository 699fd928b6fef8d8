// step_stream_fp32.cu -- cp.async streaming step kernels with float replica storage,
// one per (lanes per row G, vectors per lane VPL, prefetched neighbours NB); the
// factory maps a shape to its kernel (nullptr if not built).
#include "step_impl.cuh"

namespace qqa {

using StepFn = void (*)(const InstDesc *, const Tile *, const int32_t *, RunStatus *, int32_t);

StepFn step_stream_kernel_fp32(int G, int VPL, int NB)
{
#define QQA_CASE(g, v, nb) \
    if (G == g && VPL == v && NB == nb) return qqa_step_stream_kernel<float, g, v, nb>;
    QQA_CASE(2, 1, 4) QQA_CASE(2, 1, 8)
    QQA_CASE(4, 1, 4) QQA_CASE(4, 1, 8)
    QQA_CASE(8, 1, 4) QQA_CASE(8, 1, 8)
    QQA_CASE(16, 1, 4) QQA_CASE(16, 1, 8)
    QQA_CASE(32, 1, 4) QQA_CASE(32, 1, 8)
    QQA_CASE(32, 2, 4) QQA_CASE(32, 2, 8)
#undef QQA_CASE
    return nullptr;
}

}  // namespace qqa
