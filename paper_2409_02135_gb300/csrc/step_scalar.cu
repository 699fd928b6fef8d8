// step_scalar.cu -- step kernels for runs of one replica per instance (state
// p[n], no padding lanes), FP32 or BF16 storage, L lanes per row in the sparse
// product; the factory maps (precision, L) to its kernel (nullptr if not built).
#include "step_impl.cuh"

namespace qqa {

using StepFn = void (*)(const InstDesc *, const Tile *, const int32_t *, RunStatus *, int32_t);

StepFn step_scalar_kernel(int prec, int L)
{
#define QQA_CASE(l)                                                                                           \
    if (L == l) return prec == kFP32 ? qqa_step_scalar_kernel<float, l> : qqa_step_scalar_kernel<__nv_bfloat16, l>;
    QQA_CASE(4) QQA_CASE(8) QQA_CASE(16) QQA_CASE(32)
#undef QQA_CASE
    return nullptr;
}

}  // namespace qqa
