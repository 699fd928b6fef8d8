// step_dense_update.cu -- the update kernels of the tensor-core step (everything
// after the product A.p^t: statistics, gradient, AdamW, noise, clamp, stores,
// and the fp16 planes of the new state), one per (replica storage, lanes per
// row G, 16-byte vectors per lane VPL); the factory maps a shape to its kernel
// (nullptr if not built).
#include <cuda_fp16.h>

#include "step_impl.cuh"

namespace qqa {

// ---------------------------------------------------------------------------
// Update kernel of the tensor-core step: everything after the product, for
// 32 rows of one instance per tile, with G lanes per row over the replicas as
// in the gather kernels (the same epilogue: statistics, gradient, AdamW,
// noise, clamp, stores). Y comes from the product kernel; the new p of the 32
// rows is collected in shared memory and written as the two transposed fp16
// planes of the next step's product (consecutive threads: consecutive rows).
// ---------------------------------------------------------------------------
template <typename T, int G, int VPL>
__global__ void __launch_bounds__(256, 2) qqa_dense_update_kernel(const InstDesc *__restrict__ descs,
                                                               const Tile *__restrict__ tiles,
                                                               const int32_t *__restrict__ num_tiles_p,
                                                               RunStatus *__restrict__ status, int32_t r,
                                                               int32_t ld)
{
    constexpr int VEC = VecT<T>::N;
    constexpr int R = 32 / G;        // rows per warp at a time
    extern __shared__ float pnew[];  // [32][ld] new p of the tile's rows (ld = S_pad + 1, odd)
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int gl = lane & (G - 1), grp = lane / G;
    const unsigned gmask = (G == 32) ? 0xffffffffu : (((1u << G) - 1u) << (grp * G));
    const int rows_per_pass = (blockDim.x >> 5) * R;
    const int num_tiles = *num_tiles_p;

    for (int tile = blockIdx.x; tile < num_tiles; tile += gridDim.x) {
        const Tile tl = tiles[tile];
        const InstDesc *__restrict__ d = descs + tl.slot;
        const int t = d->t + r;
        if (t >= d->K) continue;   // block-uniform
        const StepCtx c = make_ctx(d, t, r);
        for (int base = 0; base < 32; base += rows_per_pass) {
            const int rl = base + warp * R + grp;
            const int row = tl.row0 + rl;
            if (rl >= 32 || row >= c.n) continue;   // group-uniform
            OwnRow<T, G, VPL> own;
            load_own<T, G, VPL>(d, c, row, gl, own);
            float Y[VPL][VEC];
            const float *yrow = d->dense_Y + (size_t)row * c.S_pad;
#pragma unroll
            for (int v = 0; v < VPL; ++v) {
                const int off = (v * G + gl) * VEC;
#pragma unroll
                for (int e = 0; e < VEC; ++e) Y[v][e] = 0.0f;
                if (off < c.S_pad) load_f32_vec(yrow + off, Y[v], VEC);
            }
            float dsum = 0.0f;
            if (c.kind == kMaxCut)
                dsum = row_weight_sum<G>(d, __ldg(d->row_ptr + row), __ldg(d->row_ptr + row + 1), gl, gmask);
            update_row<T, G, VPL>(d, c, row, gl, gmask, Y, dsum, own, status, pnew + (size_t)rl * ld);
        }
        __syncthreads();
        __half *XTn = reinterpret_cast<__half *>(d->dense_XT) + (size_t)((t + 1) & 1) * 2 * d->dense_N * d->n_pad;
        __half *XTn_lo = XTn + (size_t)d->dense_N * d->n_pad;
        for (int idx = threadIdx.x; idx < 32 * c.S_pad; idx += blockDim.x) {
            const int j = idx & 31, s2 = idx >> 5;
            const int row = tl.row0 + j;
            if (row < c.n) {
                const float pv = pnew[j * ld + s2];
                const __half hi = __float2half_rn(pv);
                XTn[(size_t)s2 * d->n_pad + row] = hi;
                XTn_lo[(size_t)s2 * d->n_pad + row] = __float2half_rn(pv - __half2float(hi));
            }
        }
        __syncthreads();   // pnew is rewritten by the next tile
    }
}

using UpdFn = void (*)(const InstDesc *, const Tile *, const int32_t *, RunStatus *, int32_t, int32_t);

UpdFn dense_update_kernel(int prec, int G, int VPL)
{
#define QQA_CASE_F(g, v) \
    if (prec == kFP32 && G == g && VPL == v) return qqa_dense_update_kernel<float, g, v>;
#define QQA_CASE_B(g, v) \
    if (prec != kFP32 && G == g && VPL == v) return qqa_dense_update_kernel<__nv_bfloat16, g, v>;
    QQA_CASE_F(1, 1) QQA_CASE_F(1, 2) QQA_CASE_F(1, 4) QQA_CASE_F(2, 4) QQA_CASE_F(4, 4) QQA_CASE_F(8, 4)
    QQA_CASE_F(16, 4)
    QQA_CASE_B(1, 1) QQA_CASE_B(1, 2) QQA_CASE_B(2, 2) QQA_CASE_B(4, 2) QQA_CASE_B(8, 2) QQA_CASE_B(16, 2)
#undef QQA_CASE_F
#undef QQA_CASE_B
    return nullptr;
}

}  // namespace qqa
