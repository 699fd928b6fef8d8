// step_pipe_bf16.cu -- pipelined step kernels (next tile's own rows bulk-copied to a
// shared-memory double buffer) with __nv_bfloat16 replica storage, one per (lanes per row G,
// 16-byte vectors per lane VPL); the factory maps a shape to its kernel (nullptr if
// not built).
#include "step_impl.cuh"

namespace qqa {

using PipeFn = void (*)(const InstDesc *, const Tile *, const int32_t *, RunStatus *, int32_t, int32_t);

PipeFn step_pipe_kernel_bf16(int G, int VPL, bool segs)
{
#define QQA_CASE1(g) \
    if (G == g && VPL == 1) return segs ? qqa_step_pipe_kernel_v1<__nv_bfloat16, g, true> : qqa_step_pipe_kernel_v1<__nv_bfloat16, g, false>;
#define QQA_CASE(g, v) \
    if (G == g && VPL == v) return segs ? qqa_step_pipe_kernel<__nv_bfloat16, g, v, true> : qqa_step_pipe_kernel<__nv_bfloat16, g, v, false>;
    QQA_CASE1(1) QQA_CASE(1, 2) QQA_CASE(1, 4)
    QQA_CASE1(2) QQA_CASE(2, 2) QQA_CASE(2, 4)
    QQA_CASE1(4) QQA_CASE(4, 2) QQA_CASE(4, 4)
    QQA_CASE1(8) QQA_CASE(8, 2) QQA_CASE(8, 4)
    QQA_CASE1(16) QQA_CASE(16, 2) QQA_CASE(16, 4)
    QQA_CASE1(32) QQA_CASE(32, 2) QQA_CASE(32, 4)
#undef QQA_CASE
#undef QQA_CASE1
    return nullptr;
}

}  // namespace qqa
