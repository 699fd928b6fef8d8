// step_impl.cuh -- the fused PQQA step kernel (one launch per annealing step).
//
// For every (node i, replica s) of every active instance the kernel computes,
// reading only p^t and writing p^{t+1} into the other ping-pong buffer:
//   Y      = sum_k w_k p^t[col_k][s]            CSR SpMM row, FP32 accumulate in CSR order
//   g      = MIS:    -1 + lambda Y                                (Eq. 22)
//            clique: -1 + lambda (sum_i p_is - 1/2 - Y)           (Eq. 24)
//            cut:    2 Y - d_i,  d_i = sum_k w_k                  (Eq. 26)
//   g     += gamma_t * (-2a) (2p - 1)^(a-1)                       (Eq. 7; gamma_t linear, App. C.2)
//   g     -= alpha (p - mean_i) / sqrt(var_i + eps)               (Eq. 10, population var over S)
//   AdamW  (decoupled decay, bias-corrected, Sec. 3.4 / App. C.3), + sqrt(2 lr T) xi (Eq. 11),
//   clamp to [0, 1] (Sec. 5).
//
// Layout and mapping: a group of G lanes owns one node row; lane gl of the
// group holds vectors v*G + gl (v < VPL) of the row, each 16 bytes = VEC
// replicas, so a group reads a neighbour row with VPL coalesced 128-bit loads
// per lane. Neighbour indices are loaded G at a time by the group and
// broadcast with register shuffles. Row statistics (mean, variance over the S
// replicas) are group-wide xor-shuffle reductions. Nothing is staged in
// global memory between the parts: the whole step is one kernel.
#pragma once

#include "qqa_internal.cuh"

namespace qqa {

__device__ __forceinline__ void load_f32_vec(const float *p, float *out, int n)
{
    // n = 4 or 8 contiguous floats, 16-byte aligned
    for (int k = 0; k < n; k += 4) {
        const float4 a = *reinterpret_cast<const float4 *>(p + k);
        out[k] = a.x; out[k + 1] = a.y; out[k + 2] = a.z; out[k + 3] = a.w;
    }
}

__device__ __forceinline__ void store_f32_vec(float *p, const float *in, int n)
{
    for (int k = 0; k < n; k += 4)
        *reinterpret_cast<float4 *>(p + k) = make_float4(in[k], in[k + 1], in[k + 2], in[k + 3]);
}

template <int G>
__device__ __forceinline__ float group_sum(float x, unsigned mask)
{
#pragma unroll
    for (int off = G / 2; off > 0; off >>= 1) x += __shfl_xor_sync(mask, x, off, G);
    return x;
}

// 1 - b^k computed without cancellation: -expm1(k * log1p(b - 1)); b - 1 is exact for b in [0.5, 1].
__device__ __forceinline__ float one_minus_pow(float b, int k)
{
    return -expm1f((float)k * log1pf(b - 1.0f));
}

template <typename T, int G, int VPL>
__global__ void __launch_bounds__(256) qqa_step_kernel(const InstDesc *__restrict__ descs,
                                                       const Tile *__restrict__ tiles,
                                                       const int32_t *__restrict__ num_tiles_p,
                                                       RunStatus *__restrict__ status, int32_t r)
{
    constexpr int VEC = VecT<T>::N;
    constexpr int ROWS_PER_WARP = 32 / G;
    constexpr int UNR = VPL >= 4 ? 1 : (VPL == 2 ? 2 : 4);   // neighbours in flight per batch
    extern __shared__ float sh_colsum[];

    const int lane = threadIdx.x & 31;
    const int warp = threadIdx.x >> 5;
    const int gl = lane & (G - 1);
    const int grp = lane / G;
    const unsigned gmask = (G == 32) ? 0xffffffffu : (((1u << G) - 1u) << (grp * G));
    const int num_tiles = *num_tiles_p;

    for (int tile = blockIdx.x; tile < num_tiles; tile += gridDim.x) {
        const Tile tl = tiles[tile];
        const InstDesc *__restrict__ d = descs + tl.slot;
        const int t = d->t + r;
        if (t >= d->K) continue;   // finished instance: whole block skips (same tile)

        const int n = d->n, S = d->S, S_pad = d->S_pad, kind = d->kind;
        const bool clique = (kind == kMaxClique);
        const int row = tl.row0 + warp * ROWS_PER_WARP + grp;

        // step scalars (identical in every thread of the instance)
        const float gamma = d->K > 1 ? d->gmin + (d->gmax - d->gmin) * ((float)t / (float)(d->K - 1)) : d->gmin;
        const float ent_coef = gamma * (-2.0f * (float)d->a_ent);
        const int half_pow = (d->a_ent - 2) / 2;
        const float lr = d->lr, b1 = d->b1, b2 = d->b2, adam_eps = d->adam_eps;
        const float decay = 1.0f - lr * d->wd;
        const float step_size = lr / one_minus_pow(b1, t + 1);
        const float inv_sqrt_bc2 = rsqrtf(one_minus_pow(b2, t + 1));
        const float lambda = d->lambda, alpha = d->alpha, noise_scale = d->noise_scale;

        const T *__restrict__ Xc = reinterpret_cast<const T *>(d->X[t & 1]);
        T *__restrict__ Xn = reinterpret_cast<T *>(d->X[(t + 1) & 1]);
        const float *cs_cur = nullptr;
        float *cs_next = nullptr;
        if (clique) {
            cs_cur = d->colsum + (t % 3) * S_pad;
            cs_next = d->colsum + ((t + 1) % 3) * S_pad;
            if (tl.row0 == 0) {   // the rotating buffer used by step t+1 must start at zero
                float *cs_zero = d->colsum + ((t + 2) % 3) * S_pad;
                for (int s = threadIdx.x; s < S_pad; s += blockDim.x) cs_zero[s] = 0.0f;
            }
            for (int s = threadIdx.x; s < S_pad; s += blockDim.x) sh_colsum[s] = 0.0f;
            __syncthreads();
        }

        if (row < n) {
            const size_t rbase = (size_t)row * S_pad;
            float P[VPL][VEC];
            float Y[VPL][VEC];
#pragma unroll
            for (int v = 0; v < VPL; ++v) {
                const int off = (v * G + gl) * VEC;
#pragma unroll
                for (int e = 0; e < VEC; ++e) { Y[v][e] = 0.0f; P[v][e] = 0.0f; }
                if (off < S_pad) {
                    if (d->master) load_f32_vec(d->master + rbase + off, P[v], VEC);
                    else VecT<T>::load(Xc + rbase + off, P[v]);
                }
            }

            // ---- CSR SpMM row: Y = sum_k w_k X^t[col_k] -----------------
            const int k0 = __ldg(d->row_ptr + row), k1 = __ldg(d->row_ptr + row + 1);
            const int32_t *__restrict__ colp = d->col;
            const int32_t *__restrict__ wp = d->w;
            float dsum = 0.0f;
            for (int kb = k0; kb < k1; kb += G) {
                const int myk = kb + gl;
                int jl = 0;
                float wl = 1.0f;
                if (myk < k1) {
                    jl = __ldg(colp + myk);
                    if (wp) wl = (float)__ldg(wp + myk);
                }
                const int cnt = min(G, k1 - kb);
                int q = 0;
                for (; q + UNR <= cnt; q += UNR) {
                    int j[UNR];
                    float wq[UNR];
                    float xv[UNR][VPL][VEC];
#pragma unroll
                    for (int u = 0; u < UNR; ++u) {
                        j[u] = __shfl_sync(gmask, jl, q + u, G);
                        wq[u] = wp ? __shfl_sync(gmask, wl, q + u, G) : 1.0f;
                    }
#pragma unroll
                    for (int u = 0; u < UNR; ++u)
#pragma unroll
                        for (int v = 0; v < VPL; ++v) {
                            const int off = (v * G + gl) * VEC;
                            if (off < S_pad) VecT<T>::load_ro(Xc + (size_t)j[u] * S_pad + off, xv[u][v]);
                            else {
#pragma unroll
                                for (int e = 0; e < VEC; ++e) xv[u][v][e] = 0.0f;
                            }
                        }
#pragma unroll
                    for (int u = 0; u < UNR; ++u) {
                        dsum += wq[u];
#pragma unroll
                        for (int v = 0; v < VPL; ++v)
#pragma unroll
                            for (int e = 0; e < VEC; ++e) Y[v][e] = fmaf(wq[u], xv[u][v][e], Y[v][e]);
                    }
                }
                for (; q < cnt; ++q) {
                    const int jj = __shfl_sync(gmask, jl, q, G);
                    const float ww = wp ? __shfl_sync(gmask, wl, q, G) : 1.0f;
                    dsum += ww;
#pragma unroll
                    for (int v = 0; v < VPL; ++v) {
                        const int off = (v * G + gl) * VEC;
                        if (off < S_pad) {
                            float x[VEC];
                            VecT<T>::load_ro(Xc + (size_t)jj * S_pad + off, x);
#pragma unroll
                            for (int e = 0; e < VEC; ++e) Y[v][e] = fmaf(ww, x[e], Y[v][e]);
                        }
                    }
                }
            }

            // ---- row statistics over the S replicas (Eq. 10) ----------
            float mean = 0.0f, inv_std = 0.0f;
            if (alpha != 0.0f) {
                float sum = 0.0f;
#pragma unroll
                for (int v = 0; v < VPL; ++v)
#pragma unroll
                    for (int e = 0; e < VEC; ++e)
                        if ((v * G + gl) * VEC + e < S) sum += P[v][e];
                mean = group_sum<G>(sum, gmask) / (float)S;
                float sq = 0.0f;
#pragma unroll
                for (int v = 0; v < VPL; ++v)
#pragma unroll
                    for (int e = 0; e < VEC; ++e)
                        if ((v * G + gl) * VEC + e < S) {
                            const float dl = P[v][e] - mean;
                            sq = fmaf(dl, dl, sq);
                        }
                inv_std = rsqrtf(group_sum<G>(sq, gmask) / (float)S + d->comm_eps);
            }

            // ---- gradient, AdamW, noise, clamp, store -----------------
#pragma unroll
            for (int v = 0; v < VPL; ++v) {
                const int off = (v * G + gl) * VEC;
                if (off >= S_pad) continue;
                float M[VEC], V[VEC], xi[VEC], pn[VEC];
                VecT<T>::load(reinterpret_cast<const T *>(d->m) + rbase + off, M);
                VecT<T>::load(reinterpret_cast<const T *>(d->v) + rbase + off, V);
#pragma unroll
                for (int k = 0; k < VEC / 4; ++k)
                    gauss4(d->seed_lo, d->seed_hi, (uint32_t)row, (uint32_t)((off >> 2) + k), (uint32_t)t, xi + 4 * k);
                float csv[VEC];
                if (clique) load_f32_vec(cs_cur + off, csv, VEC);
                bool bad = false;
#pragma unroll
                for (int e = 0; e < VEC; ++e) {
                    const float p = P[v][e];
                    const float y = Y[v][e];
                    float g;
                    if (kind == kMIS) g = fmaf(lambda, y, -1.0f);
                    else if (kind == kMaxCut) g = fmaf(2.0f, y, -dsum);
                    else g = fmaf(lambda, (csv[e] - 0.5f) - y, -1.0f);
                    const float u = fmaf(2.0f, p, -1.0f);
                    float upow = u;
                    const float u2 = u * u;
                    for (int k = 0; k < half_pow; ++k) upow *= u2;
                    g = fmaf(ent_coef, upow, g);
                    if (alpha != 0.0f) g = fmaf(-alpha * inv_std, p - mean, g);
                    if (d->grad_dbg) d->grad_dbg[rbase + off + e] = g;
                    const float mn = fmaf(b1, M[e], (1.0f - b1) * g);
                    const float vn = fmaf(b2, V[e], (1.0f - b2) * (g * g));
                    const float denom = fmaf(sqrtf(vn), inv_sqrt_bc2, adam_eps);
                    float q = p * decay;
                    q = fmaf(-step_size, mn / denom, q);
                    q = fmaf(noise_scale, xi[e], q);
                    bad |= !(fabsf(q) <= 3.0e38f) || !(fabsf(g) <= 3.0e38f);
                    pn[e] = fminf(fmaxf(q, 0.0f), 1.0f);
                    M[e] = mn;
                    V[e] = vn;
                }
                if (bad) atomicAdd(&status->nonfinite, 1ULL);
                VecT<T>::store(Xn + rbase + off, pn);
                if (d->master) store_f32_vec(d->master + rbase + off, pn, VEC);
                VecT<T>::store(reinterpret_cast<T *>(d->m) + rbase + off, M);
                VecT<T>::store(reinterpret_cast<T *>(d->v) + rbase + off, V);
                if (clique) {
#pragma unroll
                    for (int e = 0; e < VEC; ++e) atomicAdd(sh_colsum + off + e, pn[e]);
                }
            }
        }

        if (clique) {
            __syncthreads();
            for (int s = threadIdx.x; s < S_pad; s += blockDim.x) atomicAdd(cs_next + s, sh_colsum[s]);
            __syncthreads();
        }
    }
}

}  // namespace qqa
