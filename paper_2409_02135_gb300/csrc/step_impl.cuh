// step_impl.cuh -- the fused PQQA step kernels (one launch per annealing step).
//
// For every (node i, replica s) of every active instance a step computes,
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
// replicas) are group-wide xor-shuffle reductions.
//
// Two kernels share the per-row epilogue and differ in where neighbour rows
// come from:
//   qqa_step_kernel       gathers each neighbour row from global memory (L2);
//                         for sparse graphs, where a row is rarely reused.
//   qqa_step_tiled_kernel stages consecutive chunks of p^t in shared memory
//                         with TMA bulk copies (double-buffered, mbarrier
//                         completion) and serves every neighbour inside the
//                         chunk from there; for dense graphs, where each staged
//                         row is reused by many rows of the block.
// Both accumulate Y in ascending neighbour order, so they give bit-identical
// results.
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

// Per-(instance, step) scalars, identical in every thread working on the
// instance; the t-dependent ones come from the table the prepare kernel fills
// once per chunk of steps (entry r = step t - t_chunk_start).
struct StepCtx {
    int t, n, S, S_pad, kind, half_pow, long_thresh;
    float ent_coef, decay, step_size, inv_sqrt_bc2, lambda, alpha, noise_scale, b1, b2, adam_eps, comm_eps, inv_S;
    const float *cs_cur;   // max-clique: column sums of p^t
    float *grad_dbg;
};

static_assert(offsetof(InstDesc, lr) % 16 == 0 && offsetof(InstDesc, comm_eps) == offsetof(InstDesc, lr) + 32,
              "the hyper-parameters are read as three 16-byte vectors");

__device__ __forceinline__ StepCtx make_ctx(const InstDesc *__restrict__ d, int t, int r)
{
    StepCtx c;
    c.t = t;
    c.n = d->n;
    c.S = d->S;
    c.S_pad = d->S_pad;
    c.kind = d->kind;
    const float4 sc = d->scal[r];
    c.ent_coef = sc.x;
    c.step_size = sc.y;
    c.inv_sqrt_bc2 = sc.z;
    c.half_pow = (d->a_ent - 2) / 2;
    // (lr, wd, b1, b2), (adam_eps, gmin, gmax, alpha), (comm_eps, noise_scale, lambda, decay)
    const float4 *hp = reinterpret_cast<const float4 *>(&d->lr);
    const float4 h0 = hp[0], h1 = hp[1], h2 = hp[2];
    c.b1 = h0.z;
    c.b2 = h0.w;
    c.adam_eps = h1.x;
    c.alpha = h1.w;
    c.comm_eps = h2.x;
    c.noise_scale = h2.y;
    c.lambda = h2.z;
    c.decay = h2.w;
    c.inv_S = 1.0f / (float)c.S;
    c.long_thresh = d->hub_active ? d->long_thresh : 0x7fffffff;
    // max-clique: the column sums of p^t, formed after the previous step by the
    // column-sum kernel (a fixed summation order, so trajectories do not depend
    // on launch order)
    c.cs_cur = c.kind == kMaxClique ? d->colsum : nullptr;
    c.grad_dbg = d->grad_dbg;
    return c;
}

// Accumulate Y += w * x for one staged or global neighbour row.
template <typename T, int G, int VPL>
__device__ __forceinline__ void accumulate_row(float (&Y)[VPL][VecT<T>::N], const T *rowp, int gl, int S_pad, float w)
{
    constexpr int VEC = VecT<T>::N;
#pragma unroll
    for (int v = 0; v < VPL; ++v) {
        const int off = (v * G + gl) * VEC;
        if (off < S_pad) {
            float x[VEC];
            VecT<T>::load(rowp + off, x);
#pragma unroll
            for (int e = 0; e < VEC; ++e) Y[v][e] = fmaf(w, x[e], Y[v][e]);
        }
    }
}

// Where a row's neighbours are: its CSR range and, for the lane group's first
// batch, lane gl's neighbour index and weight (0 past the end of the row).
struct RowIdx {
    int k0, k1, jl;
    float wl;
};

__device__ __forceinline__ RowIdx load_row_idx(const InstDesc *__restrict__ d, int row, int gl)
{
    RowIdx x{0, 0, 0, 0.0f};
    if (row < d->n) {
        x.k0 = __ldg(d->row_ptr + row);
        x.k1 = __ldg(d->row_ptr + row + 1);
        if (x.k0 + gl < x.k1) {
            x.jl = __ldg(d->col + x.k0 + gl);
            x.wl = d->w ? (float)__ldg(d->w + x.k0 + gl) : 1.0f;
        }
    }
    return x;
}

// N neighbours q0..q0+N-1 of the lane group's current index batch: all loads
// in flight together, then added in CSR order. Unweighted graphs add plainly
// (exactly fmaf(1, x, y)).
template <typename T, int G, int VPL, int N, bool HINT>
__device__ __forceinline__ void gather_batch(const T *__restrict__ Xc, int jl, float wl, int q0, bool weighted,
                                             const int (&offs)[VPL], int S_pad, unsigned gmask,
                                             float (&Y)[VPL][VecT<T>::N], uint64_t pol_keep)
{
    constexpr int VEC = VecT<T>::N;
    uint4 raw[N][VPL];   // packed until accumulated: 4 registers per 16-byte slice
#pragma unroll
    for (int u = 0; u < N; ++u) {
        const T *rowp = Xc + (size_t)__shfl_sync(gmask, jl, q0 + u, G) * S_pad;
#pragma unroll
        for (int v = 0; v < VPL; ++v)
            raw[u][v] = HINT ? ld_nc_hint(rowp + offs[v], pol_keep) : __ldg(reinterpret_cast<const uint4 *>(rowp + offs[v]));
    }
#pragma unroll
    for (int u = 0; u < N; ++u) {
        const float w = weighted ? __shfl_sync(gmask, wl, q0 + u, G) : 1.0f;
#pragma unroll
        for (int v = 0; v < VPL; ++v) {
            if (!weighted) {
                VecT<T>::add_to(raw[u][v], Y[v]);
            } else {
                float xv[VEC];
                VecT<T>::unpack(raw[u][v], xv);
#pragma unroll
                for (int e = 0; e < VEC; ++e) Y[v][e] = fmaf(w, xv[e], Y[v][e]);
            }
        }
    }
}

// Y = sum of the neighbour rows of a row whose indices start in `x`.
// Neighbours go in batches of UNR whose loads are all in flight together (a
// short row costs one round trip to L2); the last, shorter batch takes
// straight-line code for its exact length. HINT: loads carry the L2 policy
// pol_keep.
template <typename T, int G, int VPL, bool HINT = false>
__device__ __forceinline__ void gather_row(const InstDesc *__restrict__ d, const T *__restrict__ Xc, const RowIdx &x,
                                           int S_pad, int gl, unsigned gmask, float (&Y)[VPL][VecT<T>::N],
                                           float &dsum, uint64_t pol_keep = 0)
{
    constexpr int VEC = VecT<T>::N;
    constexpr int UNR = VPL >= 4 ? 2 : 4;   // neighbours in flight per batch
    const int32_t *__restrict__ colp = d->col;
    const int32_t *__restrict__ wp = d->w;
    const bool weighted = wp != nullptr;
    // this lane's column offsets; lanes past the padded row read column 0 and discard it
    int offs[VPL];
    bool inr[VPL];
#pragma unroll
    for (int v = 0; v < VPL; ++v) {
        offs[v] = (v * G + gl) * VEC;
        inr[v] = offs[v] < S_pad;
        if (!inr[v]) offs[v] = 0;
    }
    if (!weighted) dsum = (float)(x.k1 - x.k0);
    int jl = x.jl;
    float wl = x.wl;
    for (int kb = x.k0; kb < x.k1; kb += G) {
        if (kb != x.k0) {   // later batches of a long row load their indices here
            const int myk = kb + gl;
            jl = 0;
            wl = 0.0f;
            if (myk < x.k1) {
                jl = __ldg(colp + myk);
                wl = weighted ? (float)__ldg(wp + myk) : 1.0f;
            }
        }
        if (weighted) dsum += group_sum<G>(wl, gmask);
        const int cnt = min(G, x.k1 - kb);
        int q = 0;
        for (; q + UNR <= cnt; q += UNR)
            gather_batch<T, G, VPL, UNR, HINT>(Xc, jl, wl, q, weighted, offs, S_pad, gmask, Y, pol_keep);
        switch (cnt - q) {   // group-uniform
            case 1: gather_batch<T, G, VPL, 1, HINT>(Xc, jl, wl, q, weighted, offs, S_pad, gmask, Y, pol_keep); break;
            case 2:
                if (UNR > 2) gather_batch<T, G, VPL, 2, HINT>(Xc, jl, wl, q, weighted, offs, S_pad, gmask, Y, pol_keep);
                break;
            case 3:
                if (UNR > 3) gather_batch<T, G, VPL, 3, HINT>(Xc, jl, wl, q, weighted, offs, S_pad, gmask, Y, pol_keep);
                break;
            default: break;
        }
    }
#pragma unroll
    for (int v = 0; v < VPL; ++v)
        if (!inr[v]) {
#pragma unroll
            for (int e = 0; e < VEC; ++e) Y[v][e] = 0.0f;
        }
}

// The row's own data: p (FP32 master or state), the AdamW moments, and the
// clique column sums. Loaded before the sparse product where registers allow,
// so their latency overlaps the neighbour gathers.
__device__ __forceinline__ uint32_t smem_addr(const void *p) { return (uint32_t)__cvta_generic_to_shared(p); }

template <typename T, int G, int VPL>
struct OwnRow {
    float P[VPL][VecT<T>::N];
    uint4 M[VPL], V[VPL];   // raw 16-byte storage vectors, unpacked when used
    static constexpr bool kLean = false;   // the whole row is in registers
    __device__ __forceinline__ void load_p(int v, float (&out)[VecT<T>::N]) const
    {
#pragma unroll
        for (int e = 0; e < VecT<T>::N; ++e) out[e] = P[v][e];
    }
    __device__ __forceinline__ uint4 mraw(int v) const { return M[v]; }
    __device__ __forceinline__ uint4 vraw(int v) const { return V[v]; }
};

// The same row read from shared memory each time a vector is used, so only
// one vector of it occupies registers at a time.
template <typename T, int G, int VPL>
struct OwnSmem {
    const float *sP;   // this row's p in shared memory
    const T *sM, *sV;  // this row's m, v in shared memory
    int gl;
    static constexpr bool kLean = true;
    __device__ __forceinline__ void load_p(int v, float (&out)[VecT<T>::N]) const
    {
        const float *q = sP + (v * G + gl) * VecT<T>::N;
#pragma unroll
        for (int k = 0; k < VecT<T>::N; k += 4) {
            float4 a;
            asm volatile("ld.shared.v4.f32 {%0, %1, %2, %3}, [%4];"
                         : "=f"(a.x), "=f"(a.y), "=f"(a.z), "=f"(a.w)
                         : "r"(smem_addr(q + k)));
            out[k] = a.x; out[k + 1] = a.y; out[k + 2] = a.z; out[k + 3] = a.w;
        }
    }
    __device__ __forceinline__ static uint4 lds16(const void *q)
    {
        uint4 a;
        asm volatile("ld.shared.v4.u32 {%0, %1, %2, %3}, [%4];" : "=r"(a.x), "=r"(a.y), "=r"(a.z), "=r"(a.w) : "r"(smem_addr(q)));
        return a;
    }
    __device__ __forceinline__ uint4 mraw(int v) const { return lds16(sM + (v * G + gl) * VecT<T>::N); }
    __device__ __forceinline__ uint4 vraw(int v) const { return lds16(sV + (v * G + gl) * VecT<T>::N); }
};

template <typename T, int G, int VPL>
__device__ __forceinline__ void load_own(const InstDesc *__restrict__ d, const StepCtx &c, int row, int gl,
                                         OwnRow<T, G, VPL> &o)
{
    constexpr int VEC = VecT<T>::N;
    const T *__restrict__ Xc = reinterpret_cast<const T *>(d->X[c.t & 1]);
    const size_t rbase = (size_t)row * c.S_pad;
#pragma unroll
    for (int v = 0; v < VPL; ++v) {
        const int off = (v * G + gl) * VEC;
#pragma unroll
        for (int e = 0; e < VEC; ++e) o.P[v][e] = 0.0f;
        o.M[v] = make_uint4(0, 0, 0, 0);
        o.V[v] = make_uint4(0, 0, 0, 0);
        if (off < c.S_pad) {
            if (d->master) {
                for (int k = 0; k < VEC; k += 4) {
                    const float4 a = *reinterpret_cast<const float4 *>(d->master + rbase + off + k);
                    o.P[v][k] = a.x; o.P[v][k + 1] = a.y; o.P[v][k + 2] = a.z; o.P[v][k + 3] = a.w;
                }
            } else {
                VecT<T>::load(Xc + rbase + off, o.P[v]);
            }
            o.M[v] = *reinterpret_cast<const uint4 *>(reinterpret_cast<const T *>(d->m) + rbase + off);
            o.V[v] = *reinterpret_cast<const uint4 *>(reinterpret_cast<const T *>(d->v) + rbase + off);
        }
    }
}

// Everything after the sparse product for one row: statistics, gradient,
// AdamW, noise, clamp, stores.
template <typename T, int G, int VPL, bool HINT = false, typename Own = OwnRow<T, G, VPL>>
__device__ __forceinline__ void update_row(const InstDesc *__restrict__ d, const StepCtx &c, int row, int gl,
                                           unsigned gmask, const float (&Y)[VPL][VecT<T>::N], float dsum,
                                           const Own &o, RunStatus *__restrict__ status, float *pn_out = nullptr,
                                           const float2 *pre_stats = nullptr, L2Policies pol = L2Policies{0, 0})
{
    constexpr int VEC = VecT<T>::N;
    T *__restrict__ Xn = reinterpret_cast<T *>(d->X[(c.t + 1) & 1]);
    const size_t rbase = (size_t)row * c.S_pad;

    // row statistics over the S replicas (Eq. 10)
    float mean = 0.0f, inv_std = 0.0f;
    if (c.alpha != 0.0f && pre_stats) {   // row statistics computed earlier by the caller
        mean = pre_stats->x;
        inv_std = pre_stats->y;
    } else if (c.alpha != 0.0f && c.S == G * VPL * VEC) {   // every lane's vectors are all replicas
        float sum = 0.0f;
#pragma unroll
        for (int v = 0; v < VPL; ++v) {
            float P[VEC];
            o.load_p(v, P);
#pragma unroll
            for (int e = 0; e < VEC; ++e) sum += P[e];
        }
        mean = group_sum<G>(sum, gmask) * c.inv_S;
        float sq = 0.0f;
#pragma unroll
        for (int v = 0; v < VPL; ++v) {
            float P[VEC];
            o.load_p(v, P);
#pragma unroll
            for (int e = 0; e < VEC; ++e) {
                const float dl = P[e] - mean;
                sq = fmaf(dl, dl, sq);
            }
        }
        inv_std = rsqrt_ftz(group_sum<G>(sq, gmask) * c.inv_S + c.comm_eps);
    } else if (c.alpha != 0.0f) {
        float sum = 0.0f;
#pragma unroll
        for (int v = 0; v < VPL; ++v) {
            const int nv = c.S - (v * G + gl) * VEC;   // valid replicas in this vector
            float P[VEC];
            o.load_p(v, P);
            if (nv >= VEC) {
#pragma unroll
                for (int e = 0; e < VEC; ++e) sum += P[e];
            } else {
#pragma unroll
                for (int e = 0; e < VEC; ++e)
                    if (e < nv) sum += P[e];
            }
        }
        mean = group_sum<G>(sum, gmask) * c.inv_S;
        float sq = 0.0f;
#pragma unroll
        for (int v = 0; v < VPL; ++v) {
            const int nv = c.S - (v * G + gl) * VEC;
            float P[VEC];
            o.load_p(v, P);
#pragma unroll
            for (int e = 0; e < VEC; ++e) {
                const float dl = P[e] - mean;
                if (nv >= VEC || e < nv) sq = fmaf(dl, dl, sq);
            }
        }
        inv_std = rsqrt_ftz(group_sum<G>(sq, gmask) * c.inv_S + c.comm_eps);
    }
    // alpha = 0 gives the coefficient -0 and adds exactly nothing
    const float comm_coef = -c.alpha * inv_std;
    // problem gradient g = A y + B for MIS (Eq. 22) and max-cut (Eq. 26)
    const float gA = c.kind == kMaxCut ? 2.0f : c.lambda;
    const float gB = c.kind == kMaxCut ? -dsum : -1.0f;
    const float om_b1 = 1.0f - c.b1, om_b2 = 1.0f - c.b2;

    // Langevin noise: all of the lane's replica quads in one lockstep Philox
    // pass when they fit in 16 registers (and the row is held in registers),
    // else one pass per vector
    constexpr bool kRowNoise = VPL * VEC <= 16;
    float xi_row[kRowNoise ? VPL : 1][VEC];
    if (kRowNoise) {
        uint32_t qs[VPL * VEC / 4];
#pragma unroll
        for (int v = 0; v < VPL; ++v)
#pragma unroll
            for (int e4 = 0; e4 < VEC; e4 += 4) qs[(v * VEC + e4) / 4] = (uint32_t)(((v * G + gl) * VEC + e4) >> 2);
        gauss_quads<VPL * VEC / 4>(d->seed_lo, d->seed_hi, (uint32_t)row, qs, (uint32_t)c.t, &xi_row[0][0]);
    }

    // The per-instance choices (problem kind, entropy exponent, gradient dump)
    // branch once per 16-byte vector, so the element loops are straight-line.
#pragma unroll
    for (int v = 0; v < VPL; ++v) {
        const int off = (v * G + gl) * VEC;
        if (off >= c.S_pad) continue;
        float P[VEC];
        o.load_p(v, P);
        float g[VEC];
        if (c.kind == kMaxClique) {   // Eq. 24, column sums of the previous step
#pragma unroll
            for (int e = 0; e < VEC; ++e) g[e] = fmaf(c.lambda, (c.cs_cur[off + e] - 0.5f) - Y[v][e], -1.0f);
        } else {
#pragma unroll
            for (int e = 0; e < VEC; ++e) g[e] = fmaf(gA, Y[v][e], gB);
        }
        // annealed entropy term gamma_t (-2a) (2p - 1)^(a - 1) (Eq. 7)
        if (c.half_pow == 1) {   // a = 4, the paper's exponent
#pragma unroll
            for (int e = 0; e < VEC; ++e) {
                const float u = fmaf(2.0f, P[e], -1.0f);
                g[e] = fmaf(c.ent_coef, u * (u * u), g[e]);
            }
        } else {
#pragma unroll
            for (int e = 0; e < VEC; ++e) {
                const float u = fmaf(2.0f, P[e], -1.0f);
                const float u2 = u * u;
                float upow = u;
                for (int k = 0; k < c.half_pow; ++k) upow *= u2;
                g[e] = fmaf(c.ent_coef, upow, g[e]);
            }
        }
        // cross-replica communication (Eq. 10)
#pragma unroll
        for (int e = 0; e < VEC; ++e) g[e] = fmaf(comm_coef, P[e] - mean, g[e]);
        if (c.grad_dbg) {
#pragma unroll
            for (int e = 0; e < VEC; ++e) c.grad_dbg[rbase + off + e] = g[e];
        }
        float xi_vec[kRowNoise ? 1 : VEC];
        if (!kRowNoise) {
            uint32_t qs[VEC / 4];
#pragma unroll
            for (int e4 = 0; e4 < VEC; e4 += 4) qs[e4 / 4] = (uint32_t)((off + e4) >> 2);
            gauss_quads<VEC / 4>(d->seed_lo, d->seed_hi, (uint32_t)row, qs, (uint32_t)c.t, xi_vec);
        }
        const float *xi = kRowNoise ? xi_row[kRowNoise ? v : 0] : xi_vec;
        float pn[VEC], M[VEC], V[VEC];
        VecT<T>::unpack(o.mraw(v), M);
        VecT<T>::unpack(o.vraw(v), V);
        float vsum = 0.0f;
#pragma unroll
        for (int e = 0; e < VEC; ++e) {
            // AdamW with decoupled decay (Sec. 3.4), noise sqrt(2 lr T) xi (Eq. 11),
            // clamp to [0, 1] (saturation; it maps NaN to 0)
            const float mn = fmaf(c.b1, M[e], om_b1 * g[e]);
            const float vn = fmaf(c.b2, V[e], om_b2 * (g[e] * g[e]));
            const float denom = fmaf(sqrt_nonneg(vn), c.inv_sqrt_bc2, c.adam_eps);
            float q = P[e] * c.decay;
            q = fmaf(-c.step_size, mn * rcp_ftz(denom), q);
            pn[e] = __saturatef(fmaf(c.noise_scale, xi[e], q));
            vsum += vn;
            M[e] = mn;
            V[e] = vn;
        }
        // p, m and v enter finite (the state is checked on the way in), so any
        // NaN, Inf or overflow of the gradient shows in the second moment
        if (!(vsum <= 3.0e38f)) atomicAdd(&status->nonfinite, 1ULL);
        if (HINT) {
            st_hint(Xn + rbase + off, VecT<T>::pack(pn), pol.keep);
            if (d->master) {
#pragma unroll
                for (int k = 0; k < VEC; k += 4)
                    st_hint(d->master + rbase + off + k, VecT<float>::pack(pn + k), pol.stream);
            }
            st_hint(reinterpret_cast<T *>(d->m) + rbase + off, VecT<T>::pack(M), pol.stream);
            st_hint(reinterpret_cast<T *>(d->v) + rbase + off, VecT<T>::pack(V), pol.stream);
        } else {
            VecT<T>::store(Xn + rbase + off, pn);
            if (d->master) {
                for (int k = 0; k < VEC; k += 4)
                    *reinterpret_cast<float4 *>(d->master + rbase + off + k) =
                        make_float4(pn[k], pn[k + 1], pn[k + 2], pn[k + 3]);
            }
            VecT<T>::store(reinterpret_cast<T *>(d->m) + rbase + off, M);
            VecT<T>::store(reinterpret_cast<T *>(d->v) + rbase + off, V);
        }
        if (pn_out) {   // new values also go to a caller buffer (the tensor-core step's plane transpose)
#pragma unroll
            for (int e = 0; e < VEC; ++e) pn_out[off + e] = pn[e];
        }
    }
}

// ---------------------------------------------------------------------------
// Direct-gather kernel: a group of G lanes per row, 256 threads per block,
// (slot, row-block) tiles walked with a grid stride.
// ---------------------------------------------------------------------------
template <typename T, int G, int VPL>
__global__ void __launch_bounds__(256) qqa_step_kernel(const InstDesc *__restrict__ descs,
                                                       const Tile *__restrict__ tiles,
                                                       const int32_t *__restrict__ num_tiles_p,
                                                       RunStatus *__restrict__ status, int32_t r)
{
    constexpr int VEC = VecT<T>::N;
    constexpr int ROWS_PER_WARP = 32 / G;

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
        const StepCtx c = make_ctx(d, t, r);
        const int row = tl.row0 + warp * ROWS_PER_WARP + grp;
        if (row < c.n) {
            const RowIdx ix = load_row_idx(d, row, gl);
            if (ix.k1 - ix.k0 > c.long_thresh) continue;   // a long row: the long-row kernel updates it
            const T *__restrict__ Xc = reinterpret_cast<const T *>(d->X[t & 1]);
            float Y[VPL][VEC];
#pragma unroll
            for (int v = 0; v < VPL; ++v)
#pragma unroll
                for (int e = 0; e < VEC; ++e) Y[v][e] = 0.0f;
            float dsum = 0.0f;
            OwnRow<T, G, VPL> own;
            constexpr bool kPrefetch = VPL <= 2;   // own row in flight during the gather
            if (kPrefetch) load_own<T, G, VPL>(d, c, row, gl, own);
            gather_row<T, G, VPL>(d, Xc, ix, c.S_pad, gl, gmask, Y, dsum);
            if (!kPrefetch) load_own<T, G, VPL>(d, c, row, gl, own);
            update_row<T, G, VPL>(d, c, row, gl, gmask, Y, dsum, own, status);
        }
    }
}

// ---------------------------------------------------------------------------
// TMA-staged kernel. Shared memory: two mbarriers, two chunk buffers of CB
// rows of p^t each, and the tile's CSR index segment. Each warp owns RPW row
// groups, so a block covers 8 * RPW * (32 / G) rows; the block streams the
// chunks that contain its rows' neighbours (from the smallest to the largest
// neighbour index) and every row consumes, per chunk, the prefix of its
// remaining (sorted) neighbour list that falls inside the chunk.
// ---------------------------------------------------------------------------

__device__ __forceinline__ void mbar_init(uint64_t *mbar, uint32_t count)
{
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_addr(mbar)), "r"(count) : "memory");
}

__device__ __forceinline__ void mbar_arrive_expect_tx(uint64_t *mbar, uint32_t bytes)
{
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_addr(mbar)), "r"(bytes)
                 : "memory");
}

__device__ __forceinline__ bool mbar_try_wait(uint64_t *mbar, uint32_t parity)
{
    uint32_t ok;
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
        "selp.u32 %0, 1, 0, p;\n\t}"
        : "=r"(ok)
        : "r"(smem_addr(mbar)), "r"(parity)
        : "memory");
    return ok != 0;
}

// Bulk (non-tensor) TMA copy global -> shared, completion counted on mbar.
// dst, src 16-byte aligned; bytes a multiple of 16.
__device__ __forceinline__ void tma_bulk_load(void *dst, const void *src, uint32_t bytes, uint64_t *mbar)
{
    asm volatile("cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
                     smem_addr(dst)),
                 "l"(src), "r"(bytes), "r"(smem_addr(mbar))
                 : "memory");
}

// The same with an L2 cache policy for the source reads.
__device__ __forceinline__ void tma_bulk_load_hint(void *dst, const void *src, uint32_t bytes, uint64_t *mbar,
                                                   uint64_t pol)
{
    asm volatile(
        "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes.L2::cache_hint [%0], [%1], %2, [%3], %4;" ::"r"(
            smem_addr(dst)),
        "l"(src), "r"(bytes), "r"(smem_addr(mbar)), "l"(pol)
        : "memory");
}

// Wait for phase `parity` of mbar with a clock limit; false if it ran out.
// (The clock is read only once the phase is found incomplete.)
__device__ __forceinline__ bool mbar_wait_bounded(uint64_t *mbar, uint32_t parity)
{
    if (mbar_try_wait(mbar, parity)) return true;
    const long long start = clock64();
    while (!mbar_try_wait(mbar, parity)) {
        if (clock64() - start > (1LL << 31)) return false;   // ~1 s at 2 GHz
    }
    return true;
}

struct TiledSmem {
    uint64_t mbar[2];
    int32_t lo, hi;
    int32_t pad[2];
};

// Capacity (ints) of the shared-memory copy of a tile's CSR index segment.
constexpr int kTiledIdxCap = 8192;

template <typename T, int G, int VPL, int RPW>
__global__ void __launch_bounds__(256) qqa_step_tiled_kernel(const InstDesc *__restrict__ descs,
                                                             const Tile *__restrict__ tiles,
                                                             const int32_t *__restrict__ num_tiles_p,
                                                             RunStatus *__restrict__ status, int32_t r,
                                                             int32_t chunk_rows, int32_t buf_elems)
{
    constexpr int VEC = VecT<T>::N;
    constexpr int GPW = 32 / G;   // row groups per warp
    extern __shared__ __align__(128) unsigned char smem_raw[];
    TiledSmem *hdr = reinterpret_cast<TiledSmem *>(smem_raw);
    T *buf0 = reinterpret_cast<T *>(smem_raw + 128);
    T *bufs[2] = {buf0, buf0 + buf_elems};
    int32_t *sidx = reinterpret_cast<int32_t *>(buf0 + 2 * (size_t)buf_elems);

    const int lane = threadIdx.x & 31;
    const int warp = threadIdx.x >> 5;
    const int gl = lane & (G - 1);
    const int grp = lane / G;
    const unsigned gmask = (G == 32) ? 0xffffffffu : (((1u << G) - 1u) << (grp * G));
    const int rows_per_block = (blockDim.x >> 5) * RPW * GPW;
    const int num_tiles = *num_tiles_p;

    if (threadIdx.x == 0) {
        mbar_init(&hdr->mbar[0], 1);
        mbar_init(&hdr->mbar[1], 1);
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    __syncthreads();
    uint32_t uses0 = 0, uses1 = 0;   // completed phases of each buffer's barrier (block-uniform)

    for (int tile = blockIdx.x; tile < num_tiles; tile += gridDim.x) {
        const Tile tl = tiles[tile];
        const InstDesc *__restrict__ d = descs + tl.slot;
        const int t = d->t + r;
        if (t >= d->K) continue;
        const StepCtx c = make_ctx(d, t, r);
        const T *__restrict__ Xc = reinterpret_cast<const T *>(d->X[t & 1]);
        const int32_t *__restrict__ colp = d->col;
        const int32_t *__restrict__ wp = d->w;
        const size_t row_bytes = (size_t)c.S_pad * sizeof(T);

        // neighbour range of the block's rows -> chunks to stream
        if (threadIdx.x == 0) { hdr->lo = 0x7fffffff; hdr->hi = -1; }
        __syncthreads();
        int kcur[RPW], kend[RPW];
        float dsum[RPW];
        float Y[RPW][VPL][VEC];
#pragma unroll
        for (int q = 0; q < RPW; ++q) {
            const int row = tl.row0 + (warp * RPW + q) * GPW + grp;
            kcur[q] = 0;
            kend[q] = 0;
            dsum[q] = 0.0f;
            if (row < c.n) {
                kcur[q] = __ldg(d->row_ptr + row);
                kend[q] = __ldg(d->row_ptr + row + 1);
                if (kend[q] - kcur[q] > c.long_thresh) kcur[q] = kend[q];   // long row: updated by the long-row kernel
                if (wp == nullptr) dsum[q] = (float)(kend[q] - kcur[q]);
                if (gl == 0 && kend[q] > kcur[q]) {
                    atomicMin(&hdr->lo, __ldg(colp + kcur[q]));
                    atomicMax(&hdr->hi, __ldg(colp + kend[q] - 1));
                }
            }
#pragma unroll
            for (int v = 0; v < VPL; ++v)
#pragma unroll
                for (int e = 0; e < VEC; ++e) Y[q][v][e] = 0.0f;
        }
        // the tile's CSR index segment, copied to shared memory when it fits
        const int seg0 = __ldg(d->row_ptr + tl.row0);
        const int seg1 = __ldg(d->row_ptr + min(tl.row0 + rows_per_block, c.n));
        const bool staged_idx = wp == nullptr && seg1 - seg0 <= kTiledIdxCap;
        if (staged_idx)
            for (int k = threadIdx.x; k < seg1 - seg0; k += blockDim.x) sidx[k] = __ldg(colp + seg0 + k);
        __syncthreads();
        const int lo = hdr->lo, hi = hdr->hi;
        const int c_first = hi >= 0 ? lo / chunk_rows : 0;
        const int nch = hi >= 0 ? hi / chunk_rows - c_first + 1 : 0;

        auto issue = [&](int ci, int b) {
            const int node0 = (c_first + ci) * chunk_rows;
            const int rows = min(chunk_rows, c.n - node0);
            const uint32_t bytes = (uint32_t)(rows * row_bytes);
            mbar_arrive_expect_tx(&hdr->mbar[b], bytes);
            tma_bulk_load(bufs[b], Xc + (size_t)node0 * c.S_pad, bytes, &hdr->mbar[b]);
        };
        if (threadIdx.x == 0) {
            asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
            for (int b = 0; b < 2 && b < nch; ++b) issue(b, b);
        }
        bool failed = false;
        for (int ci = 0; ci < nch; ++ci) {
            const int b = ci & 1;
            const uint32_t parity = (b == 0 ? uses0 : uses1) & 1u;
            const bool ok = mbar_wait_bounded(&hdr->mbar[b], parity);
            if (__syncthreads_or(!ok)) { failed = true; break; }
            if (b == 0) ++uses0; else ++uses1;
            const int node0 = (c_first + ci) * chunk_rows;
            const int node_end = node0 + chunk_rows;
            const T *sb = bufs[b];
            if (staged_idx) {
                // indices from shared memory (broadcast reads), four at a time while
                // the fourth is still inside the chunk (rows are sorted)
#pragma unroll
                for (int q = 0; q < RPW; ++q) {
                    int k = kcur[q];
                    const int ke = kend[q];
                    while (k + 4 <= ke) {
                        const int j0 = sidx[k - seg0], j1 = sidx[k + 1 - seg0];
                        const int j2 = sidx[k + 2 - seg0], j3 = sidx[k + 3 - seg0];
                        if (j3 >= node_end) break;
                        accumulate_row<T, G, VPL>(Y[q], sb + (size_t)(j0 - node0) * c.S_pad, gl, c.S_pad, 1.0f);
                        accumulate_row<T, G, VPL>(Y[q], sb + (size_t)(j1 - node0) * c.S_pad, gl, c.S_pad, 1.0f);
                        accumulate_row<T, G, VPL>(Y[q], sb + (size_t)(j2 - node0) * c.S_pad, gl, c.S_pad, 1.0f);
                        accumulate_row<T, G, VPL>(Y[q], sb + (size_t)(j3 - node0) * c.S_pad, gl, c.S_pad, 1.0f);
                        k += 4;
                    }
                    while (k < ke) {
                        const int j = sidx[k - seg0];
                        if (j >= node_end) break;
                        accumulate_row<T, G, VPL>(Y[q], sb + (size_t)(j - node0) * c.S_pad, gl, c.S_pad, 1.0f);
                        ++k;
                    }
                    kcur[q] = k;
                }
            } else {
#pragma unroll
                for (int q = 0; q < RPW; ++q) {
                    int k = kcur[q];
                    const int ke = kend[q];
                    while (k < ke) {   // group-uniform loop
                        const int myk = k + gl;
                        int jl = 0x7fffffff;
                        float wl = 1.0f;
                        if (myk < ke) {
                            jl = __ldg(colp + myk);
                            if (wp) wl = (float)__ldg(wp + myk);
                        }
                        const unsigned in = __ballot_sync(gmask, jl < node_end);
                        const int cnt = __popc(G == 32 ? in : ((in >> (grp * G)) & ((1u << G) - 1u)));
                        for (int u = 0; u < cnt; ++u) {
                            const int j = __shfl_sync(gmask, jl, u, G);
                            const float w = wp ? __shfl_sync(gmask, wl, u, G) : 1.0f;
                            if (wp) dsum[q] += w;
                            accumulate_row<T, G, VPL>(Y[q], sb + (size_t)(j - node0) * c.S_pad, gl, c.S_pad, w);
                        }
                        k += cnt;
                        if (cnt < G) break;
                    }
                    kcur[q] = k;
                }
            }
            __syncthreads();   // every thread is done with buffer b
            if (threadIdx.x == 0 && ci + 2 < nch) {
                asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
                issue(ci + 2, b);
            }
        }
        if (failed) {
            // a staged copy did not arrive in time: flag it, let any copy still
            // in flight land (bounded), and leave without touching the state
            if (threadIdx.x == 0) {
                atomicAdd(&status->timeouts, 1ULL);
                mbar_wait_bounded(&hdr->mbar[0], uses0 & 1u);
                mbar_wait_bounded(&hdr->mbar[1], uses1 & 1u);
            }
            __syncthreads();
            return;
        }
#pragma unroll
        for (int q = 0; q < RPW; ++q) {
            const int row = tl.row0 + (warp * RPW + q) * GPW + grp;
            if (row < c.n && __ldg(d->row_ptr + row + 1) - __ldg(d->row_ptr + row) <= c.long_thresh) {
                OwnRow<T, G, VPL> own;
                load_own<T, G, VPL>(d, c, row, gl, own);
                update_row<T, G, VPL>(d, c, row, gl, gmask, Y[q], dsum[q], own, status);
            }
        }
        __syncthreads();   // hdr->lo / hi and sidx are rewritten by the next tile
    }
}

// ---------------------------------------------------------------------------
// Warp-pipelined kernel for sparse graphs. A tile is the 32 / G consecutive
// rows of one warp (one row per lane group), so its own data (p^t - the FP32
// master in BF16 runs -, m and v) are three contiguous slabs. Every warp walks
// its own tiles and owns a double buffer in shared memory: while it gathers
// and updates one tile, lane 0 has the next tile's three slabs in flight to the
// other buffer (bulk copies, completion counted on that buffer's mbarrier).
// The HBM latency of the streamed state is hidden without registers, and with
// no block-wide barriers the warps of an SM drift apart, so one warp's gather
// latency is covered by the others' epilogues.
// ---------------------------------------------------------------------------
// One lane group's segment partial P (FP32) of a long row: store it, and
// announce it on the row's arrival counter. The group that brings the count to
// the row's number of segments sums the partials in segment order into Y
// (Y = ((P_0 + P_1) + P_2) + ...), resets the counter for the next step and
// returns true; every other group returns false. No group waits for another.
template <typename T, int G, int VPL>
__device__ __forceinline__ bool seg_arrive(const InstDesc *__restrict__ d, int seg, int j, int s0, int s1, int gl,
                                           unsigned gmask, float (&Y)[VPL][VecT<T>::N])
{
    constexpr int VEC = VecT<T>::N;
    const int S_pad = d->S_pad;
    float *part = d->seg_part + (size_t)seg * S_pad;
#pragma unroll
    for (int v = 0; v < VPL; ++v) {
        const int off = (v * G + gl) * VEC;
        if (off < S_pad) store_f32_vec(part + off, Y[v], VEC);
    }
    __threadfence();   // this lane's partial is visible before the group announces it
    __syncwarp(gmask);
    unsigned prev = 0;
    if (gl == 0) prev = atomicAdd(d->seg_cnt + j, 1u);
    prev = __shfl_sync(gmask, prev, 0, G);
    if (prev != (unsigned)(s1 - s0 - 1)) return false;   // not the last segment of the row
    __threadfence();
    // the partials in segment order, read from L2 (other SMs wrote them in this launch)
    for (int q = s0; q < s1; ++q) {
        const float *pp = d->seg_part + (size_t)q * S_pad;
#pragma unroll
        for (int v = 0; v < VPL; ++v) {
            const int off = (v * G + gl) * VEC;
            if (off < S_pad) {
#pragma unroll
                for (int k = 0; k < VEC; k += 4) {
                    const float4 a = __ldcg(reinterpret_cast<const float4 *>(pp + off + k));
                    if (q == s0) {
                        Y[v][k] = a.x; Y[v][k + 1] = a.y; Y[v][k + 2] = a.z; Y[v][k + 3] = a.w;
                    } else {
                        Y[v][k] += a.x; Y[v][k + 1] += a.y; Y[v][k + 2] += a.z; Y[v][k + 3] += a.w;
                    }
                }
            }
        }
    }
    if (gl == 0) d->seg_cnt[j] = 0u;   // ready for the next step (a later launch)
    return true;
}

// Weighted degree sum_k w_k of a row (its neighbour count when unweighted);
// integer weights, so the sum is exact in any order.
template <int G>
__device__ __forceinline__ float row_weight_sum(const InstDesc *__restrict__ d, int k0, int k1, int gl, unsigned gmask)
{
    if (!d->w) return (float)(k1 - k0);
    float ws = 0.0f;
    for (int k = k0 + gl; k < k1; k += G) ws += (float)__ldg(d->w + k);
    return group_sum<G>(ws, gmask);
}

template <typename T, int G, int VPL>
__device__ __forceinline__ void load_own_smem(const unsigned char *buf, int R, int S_pad, int lrow, int gl,
                                              OwnRow<T, G, VPL> &o)
{
    constexpr int VEC = VecT<T>::N;
    const float *sP = reinterpret_cast<const float *>(buf) + (size_t)lrow * S_pad;
    const T *sM = reinterpret_cast<const T *>(buf + (size_t)R * S_pad * sizeof(float)) + (size_t)lrow * S_pad;
    const T *sV = sM + (size_t)R * S_pad;
#pragma unroll
    for (int v = 0; v < VPL; ++v) {
        const int off = (v * G + gl) * VEC;
#pragma unroll
        for (int e = 0; e < VEC; ++e) o.P[v][e] = 0.0f;
        o.M[v] = make_uint4(0, 0, 0, 0);
        o.V[v] = make_uint4(0, 0, 0, 0);
        if (off < S_pad) {
#pragma unroll
            for (int k = 0; k < VEC; k += 4) {
                const float4 a = *reinterpret_cast<const float4 *>(sP + off + k);
                o.P[v][k] = a.x; o.P[v][k + 1] = a.y; o.P[v][k + 2] = a.z; o.P[v][k + 3] = a.w;
            }
            o.M[v] = *reinterpret_cast<const uint4 *>(sM + off);
            o.V[v] = *reinterpret_cast<const uint4 *>(sV + off);
        }
    }
}

// SEGS: the tile list may hold segment work items of long rows (runs without
// long rows take the variant without that path). The body of the pipelined
// kernels below.
template <typename T, int G, int VPL, bool SEGS>
__device__ __forceinline__ void pipe_step(const InstDesc *__restrict__ descs, const Tile *__restrict__ tiles,
                                          const int32_t *__restrict__ num_tiles_p, RunStatus *__restrict__ status,
                                          int32_t r, int32_t buf_bytes)
{
    constexpr int R = 32 / G;   // rows of a tile: one per lane group of the warp
    extern __shared__ __align__(128) unsigned char smem_raw[];
    const int lane = threadIdx.x & 31;
    const int warp = threadIdx.x >> 5;
    const int gl = lane & (G - 1);
    const int grp = lane / G;
    const unsigned gmask = (G == 32) ? 0xffffffffu : (((1u << G) - 1u) << (grp * G));
    const int nwarps = blockDim.x >> 5;
    // header: two barriers per warp (at most 8 warps); then each warp's two buffers
    uint64_t *mbar = reinterpret_cast<uint64_t *>(smem_raw) + 2 * warp;
    unsigned char *const buf0 = smem_raw + 128 + (size_t)warp * 2 * buf_bytes;   // buffer b at buf0 + b * buf_bytes
    const int num_tiles = num_tiles_p[0];
    // num_tiles_p[1] != 0: the run's state does not fit in L2, so the streamed
    // slabs are read and written evict-first and p is kept (evict-last)
    const L2Policies pol = make_l2_policies(num_tiles_p[1] != 0);
    const int W = gridDim.x * nwarps;
    const int first = blockIdx.x * nwarps + warp;

    if (lane == 0) {
        mbar_init(&mbar[0], 1);
        mbar_init(&mbar[1], 1);
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    __syncwarp();

    // Whole warp: start the copies of tile tl's slabs into buffer b (nothing for
    // a finished instance, whose tile the warp skips, or for segment work);
    // lanes 0, 1, 2 issue the copies of p, m and v side by side. Returns
    // whether it did.
    // The step context of the instance of the previous tile (most consecutive
    // tiles of a warp belong to the same instance), with what the next tile's
    // copies, indices and prefetches need from it: this lane's copy source
    // (lanes 0, 1, 2: p, m, v), its cache policy and the gather base p^t, so
    // that a tile of the same instance reads nothing from its descriptor.
    const unsigned char *my_slab = nullptr;
    const void *xcur = nullptr;
    uint64_t my_hint = 0;
    int ctx_slot = -1;
    // With one vector per lane the step scalars of the current instance live
    // in shared memory (one copy per warp) rather than in registers, which
    // lets the register-capped variant run without spills (BA(4) max-cut
    // 157.4 -> 149.3 us at 96 registers); with more vectors per lane they stay
    // in registers (3-regular max-cut measured 0.5% slower from shared memory).
    constexpr bool kCtxShared = VPL == 1;
    __shared__ StepCtx ctx_sm[kCtxShared ? 8 : 1];   // at most 8 warps per block
    StepCtx ctx_reg{};
    StepCtx &c = kCtxShared ? ctx_sm[warp] : ctx_reg;
    auto issue = [&](const Tile &tl, int b) -> bool {
        if (SEGS && tl.row0 < 0) return false;   // segments of long rows: no slabs
        int S_pad, n;
        const unsigned char *base;
        uint64_t hint;
        if (tl.slot == ctx_slot) {
            S_pad = c.S_pad;
            n = c.n;
            base = my_slab;
            hint = my_hint;
        } else {
            const InstDesc *__restrict__ d = descs + tl.slot;
            const int t = d->t + r;
            if (t >= d->K) return false;
            S_pad = d->S_pad;
            n = d->n;
            if (lane == 0) base = reinterpret_cast<const unsigned char *>(d->master ? d->master : reinterpret_cast<const float *>(d->X[t & 1]));
            else base = reinterpret_cast<const unsigned char *>(lane == 1 ? d->m : d->v);
            hint = (lane == 0 && !d->master) ? pol.keep : pol.stream;
        }
        const int rows = min(R, n - tl.row0);
        const size_t e0 = (size_t)tl.row0 * S_pad;
        const uint32_t pbytes = (uint32_t)(rows * S_pad * sizeof(float));
        const uint32_t sbytes = (uint32_t)(rows * S_pad * sizeof(T));
        if (lane == 0) mbar_arrive_expect_tx(&mbar[b], pbytes + 2 * sbytes);
        __syncwarp();   // the expected bytes are registered before any copy can land
        if (lane < 3) {
            const size_t mofs = (size_t)R * S_pad * sizeof(float);
            const size_t vofs = mofs + (size_t)R * S_pad * sizeof(T);
            unsigned char *dst = buf0 + (size_t)b * buf_bytes + (lane == 0 ? 0 : (lane == 1 ? mofs : vofs));
            const void *src = base + e0 * (lane == 0 ? sizeof(float) : sizeof(T));
            asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
            tma_bulk_load_hint(dst, src, lane == 0 ? pbytes : sbytes, &mbar[b], hint);
        }
        return true;
    };
    // with one vector per lane there are registers to spare for the context
    // slot's CSR pointers too (measured: they help there and cost at VPL = 2)
    constexpr bool kCacheCsr = VPL == 1;
    const int32_t *rp_c = nullptr, *col_c = nullptr, *w_c = nullptr;
    auto tile_idx = [&](const Tile &tl) -> RowIdx {
        if (SEGS && tl.row0 < 0) return RowIdx{0, 0, 0, 0.0f};
        if (!kCacheCsr || tl.slot != ctx_slot) return load_row_idx(descs + tl.slot, tl.row0 + grp, gl);
        const int row = tl.row0 + grp;
        RowIdx x{0, 0, 0, 0.0f};
        if (row < c.n) {
            x.k0 = __ldg(rp_c + row);
            x.k1 = __ldg(rp_c + row + 1);
            if (x.k0 + gl < x.k1) {
                x.jl = __ldg(col_c + x.k0 + gl);
                x.wl = w_c ? (float)__ldg(w_c + x.k0 + gl) : 1.0f;
            }
        }
        return x;
    };

    // Software pipeline over the warp's tiles: tile records are fetched two
    // tiles ahead, the row bounds and first neighbour indices one tile ahead,
    // the slabs one tile ahead, and the next tile's first neighbour rows are
    // prefetched into L1 during this tile's update, so little of a tile's
    // memory latency is exposed. Segment work items of long rows (listed
    // first) take the long-row kernel's steps inside this loop: each lane group
    // sums one segment into its partial row, and the group that completes a
    // row copies the row's own state into the warp's free buffer and updates
    // it like any other row.
    const Tile none{0, 0};
    Tile tl_cur = first < num_tiles ? tiles[first] : none;
    Tile tl_nxt = first + W < num_tiles ? tiles[first + W] : none;
    RowIdx ix_cur = first < num_tiles ? tile_idx(tl_cur) : RowIdx{0, 0, 0, 0.0f};

    // completed phases of each buffer's barrier, and whether a copy is in
    // flight into the buffer not being read (warp-uniform)
    uint32_t uses0 = 0u, uses1 = 0u;
    bool next_pending = false;
    int b = 0;
    if (first < num_tiles) issue(tl_cur, 0);
    for (int tile = first; tile < num_tiles; tile += W, b ^= 1) {
        const bool has_next = tile + W < num_tiles;
        // buffer b^1 was last read in the previous iteration, which ended in __syncwarp
        next_pending = has_next && issue(tl_nxt, b ^ 1);
        RowIdx ix_nxt{0, 0, 0, 0.0f};
        if (has_next) ix_nxt = tile_idx(tl_nxt);
        const Tile tl_nn = tile + 2 * W < num_tiles ? tiles[tile + 2 * W] : none;

        const Tile tl = tl_cur;
        const RowIdx ix = ix_cur;
        tl_cur = tl_nxt;
        tl_nxt = tl_nn;
        ix_cur = ix_nxt;
        const InstDesc *__restrict__ d = descs + tl.slot;
        if (tl.slot != ctx_slot) {
            const int t = d->t + r;
            if (t >= d->K) continue;   // finished instance: no copy was issued, nothing is read
            if (kCtxShared) {
                if (lane == 0) c = make_ctx(d, t, r);
                __syncwarp();   // the warp's lanes read it below
            } else {
                c = make_ctx(d, t, r);
            }
            ctx_slot = tl.slot;
            xcur = d->X[t & 1];
            if (lane == 0) my_slab = reinterpret_cast<const unsigned char *>(d->master ? d->master : reinterpret_cast<const float *>(d->X[t & 1]));
            else my_slab = reinterpret_cast<const unsigned char *>(lane == 1 ? d->m : d->v);
            my_hint = (lane == 0 && !d->master) ? pol.keep : pol.stream;
            if (kCacheCsr) {
                rp_c = d->row_ptr;
                col_c = d->col;
                w_c = d->w;
            }
        }
        const T *__restrict__ Xc = reinterpret_cast<const T *>(xcur);
        unsigned char *const bb = buf0 + (size_t)b * buf_bytes;
        const bool segs = SEGS && tl.row0 < 0;
        float Y[VPL][VecT<T>::N];
#pragma unroll
        for (int v = 0; v < VPL; ++v)
#pragma unroll
            for (int e = 0; e < VecT<T>::N; ++e) Y[v][e] = 0.0f;
        float dsum = 0.0f;
        int row = tl.row0 + grp;
        bool mine = false;
        if (!segs) {
            // a long row is updated by its segment items (its slab rows are copied all the same)
            mine = row < c.n && ix.k1 - ix.k0 <= c.long_thresh;
            if (mine) gather_row<T, G, VPL, true>(d, Xc, ix, c.S_pad, gl, gmask, Y, dsum, pol.keep);
        } else {
            const int seg = seg_item_first(tl.row0) + grp;
            if (seg < d->nseg) {   // group-uniform
                const int j = __ldg(d->seg_row + seg);
                const int s0 = __ldg(d->seg_ptr + j), s1 = __ldg(d->seg_ptr + j + 1);
                row = __ldg(d->long_rows + j);
                const int rk0 = __ldg(d->row_ptr + row), rk1 = __ldg(d->row_ptr + row + 1);
                RowIdx x{0, 0, 0, 0.0f};
                x.k0 = rk0 + (seg - s0) * kSegLen;
                x.k1 = min(x.k0 + kSegLen, rk1);
                if (x.k0 + gl < x.k1) {
                    x.jl = __ldg(d->col + x.k0 + gl);
                    x.wl = d->w ? (float)__ldg(d->w + x.k0 + gl) : 1.0f;
                }
                gather_row<T, G, VPL, true>(d, Xc, x, c.S_pad, gl, gmask, Y, dsum, pol.keep);
                mine = seg_arrive<T, G, VPL>(d, seg, j, s0, s1, gl, gmask, Y);
                if (mine) {
                    dsum = row_weight_sum<G>(d, rk0, rk1, gl, gmask);
                    // the row's own p (FP32; the master in BF16 runs), m and v into
                    // this group's row of the free buffer, where the update reads them
                    constexpr int VEC = VecT<T>::N;
                    const size_t rb = (size_t)row * c.S_pad;
                    const float *gp = d->master ? d->master + rb : reinterpret_cast<const float *>(Xc) + rb;
                    float *sp = reinterpret_cast<float *>(bb) + (size_t)grp * c.S_pad;
                    T *sm = reinterpret_cast<T *>(bb + (size_t)R * c.S_pad * sizeof(float)) + (size_t)grp * c.S_pad;
                    T *sv = sm + (size_t)R * c.S_pad;
#pragma unroll
                    for (int v = 0; v < VPL; ++v) {
                        const int off = (v * G + gl) * VEC;
                        if (off < c.S_pad) {
#pragma unroll
                            for (int k = 0; k < VEC; k += 4)
                                *reinterpret_cast<float4 *>(sp + off + k) = *reinterpret_cast<const float4 *>(gp + off + k);
                            *reinterpret_cast<uint4 *>(sm + off) =
                                *reinterpret_cast<const uint4 *>(reinterpret_cast<const T *>(d->m) + rb + off);
                            *reinterpret_cast<uint4 *>(sv + off) =
                                *reinterpret_cast<const uint4 *>(reinterpret_cast<const T *>(d->v) + rb + off);
                        }
                    }
                    __syncwarp(gmask);
                }
            }
        }
        // the next tile's first neighbour rows (one per lane of the group, up to
        // G of them) are pulled from L2 into L1 while this tile is updated, so
        // its gather finds them there; its row bounds and first indices were
        // requested before this tile's gather. With one vector per lane (one
        // row per warp, five blocks per SM) the L1 is shared by more warps and
        // the prefetch measured slower, so that variant leaves it out.
        if (VPL != 1 && has_next && ix_cur.k0 + gl < ix_cur.k1) {
            const void *xn = xcur;
            int spn = c.S_pad;
            bool live = true;
            if (tl_cur.slot != ctx_slot) {
                const InstDesc *__restrict__ dn = descs + tl_cur.slot;
                const int tn = dn->t + r;
                live = tn < dn->K;
                xn = dn->X[tn & 1];
                spn = dn->S_pad;
            }
            if (live) {
                const char *src = reinterpret_cast<const char *>(reinterpret_cast<const T *>(xn) + (size_t)ix_cur.jl * spn);
                const int bytes = spn * (int)sizeof(T);
                for (int o = 0; o < bytes; o += 128) asm volatile("prefetch.global.L1 [%0];" ::"l"(src + o));
            }
        }
        if (!segs) {   // the slabs of this tile (segment items copied none)
            const uint32_t parity = (b ? uses1 : uses0) & 1u;
            const bool ok = __all_sync(0xffffffffu, mbar_wait_bounded(&mbar[b], parity));
            if (!ok) {
                // the slabs did not arrive in time: flag it, let every copy still in
                // flight land (bounded), and leave without touching the state
                if (lane == 0) {
                    atomicAdd(&status->timeouts, 1ULL);
                    if (next_pending) mbar_wait_bounded(&mbar[b ^ 1], (b ? uses0 : uses1) & 1u);
                    mbar_wait_bounded(&mbar[b], parity);
                }
                __syncwarp();
                return;
            }
            if (b) ++uses1; else ++uses0;
        }
        if (mine) {
            const T *sM = reinterpret_cast<const T *>(bb + (size_t)R * c.S_pad * sizeof(float)) + (size_t)grp * c.S_pad;
            const OwnSmem<T, G, VPL> own{reinterpret_cast<const float *>(bb) + (size_t)grp * c.S_pad, sM,
                                          sM + (size_t)R * c.S_pad, gl};
            update_row<T, G, VPL, true>(d, c, row, gl, gmask, Y, dsum, own, status, nullptr, nullptr, pol);
        }
        __syncwarp();   // every lane is done with buffer b
    }
}

template <typename T, int G, int VPL, bool SEGS>
__global__ void __launch_bounds__(256) qqa_step_pipe_kernel(const InstDesc *__restrict__ descs,
                                                            const Tile *__restrict__ tiles,
                                                            const int32_t *__restrict__ num_tiles_p,
                                                            RunStatus *__restrict__ status, int32_t r,
                                                            int32_t buf_bytes)
{
    pipe_step<T, G, VPL, SEGS>(descs, tiles, num_tiles_p, status, r, buf_bytes);
}

// With one vector per lane (and the step scalars in shared memory) the kernel
// is held to 80 registers without spills, so that six blocks of 128 threads
// fit on an SM instead of four: more warps hide more of the dependent gather
// latency (BA(4) max-cut n = 1e5: 157.4 us at 127 registers, 149.3 at 96,
// 138.4 at 80; 72 registers spill and measured 139.5).
template <typename T, int G, bool SEGS>
__global__ void __maxnreg__(80) qqa_step_pipe_kernel_v1(const InstDesc *__restrict__ descs,
                                                        const Tile *__restrict__ tiles,
                                                        const int32_t *__restrict__ num_tiles_p,
                                                        RunStatus *__restrict__ status, int32_t r,
                                                        int32_t buf_bytes)
{
    pipe_step<T, G, 1, SEGS>(descs, tiles, num_tiles_p, status, r, buf_bytes);
}

// ---------------------------------------------------------------------------
// Streaming kernel for sparse graphs: each thread keeps a private, double-
// buffered prefetch area in shared memory. While it computes row i it has
// already asked, with cp.async (16 bytes per request, L2-only caching), for
// exactly the 16-byte slices of row i+1 it will need: its own p (FP32 master or
// state), m and v, and the slices of the first NB neighbour rows. Completion is
// tracked per thread by cp.async.wait_group, so no barrier or spin-wait is
// involved; neighbours beyond NB are gathered directly, after the prefetched
// ones, which keeps the ascending accumulation order of the other kernels.
// ---------------------------------------------------------------------------
__device__ __forceinline__ void cp_async16(void *smem_dst, const void *gmem_src)
{
    asm volatile("cp.async.cg.shared.global [%0], [%1], 16;" ::"r"(smem_addr(smem_dst)), "l"(gmem_src) : "memory");
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;" ::: "memory"); }
__device__ __forceinline__ void cp_async_wait_1() { asm volatile("cp.async.wait_group 1;" ::: "memory"); }

struct StreamItem {
    const InstDesc *d;
    int row, t, k0, k1;
    bool exists, valid;
};

template <typename T, int G, int VPL, int NB>
__global__ void __launch_bounds__(256) qqa_step_stream_kernel(const InstDesc *__restrict__ descs,
                                                              const Tile *__restrict__ tiles,
                                                              const int32_t *__restrict__ num_tiles_p,
                                                              RunStatus *__restrict__ status, int32_t r)
{
    constexpr int VEC = VecT<T>::N;
    constexpr int GPW = 32 / G;
    constexpr int PW = sizeof(T) == 2 ? 2 : 1;   // 16-byte words of the own p slice (FP32 master for BF16)
    constexpr int SLOTS = PW + 2 + NB;          // p, m, v, neighbours
    extern __shared__ uint4 sh_pf[];            // [2][VPL][SLOTS][blockDim]

    const int lane = threadIdx.x & 31;
    const int warp = threadIdx.x >> 5;
    const int gl = lane & (G - 1);
    const int grp = lane / G;
    const unsigned gmask = (G == 32) ? 0xffffffffu : (((1u << G) - 1u) << (grp * G));
    const int num_tiles = *num_tiles_p;
    const int nthr = blockDim.x;
    auto slot_ptr = [&](int stage, int v, int slot) -> uint4 * {
        return sh_pf + ((size_t)((stage * VPL + v) * SLOTS + slot)) * nthr + threadIdx.x;
    };

    auto fetch = [&](int it) -> StreamItem {
        StreamItem x;
        const int tile = blockIdx.x + it * gridDim.x;
        x.exists = tile < num_tiles;
        x.valid = false;
        x.d = nullptr;
        x.row = x.t = x.k0 = x.k1 = 0;
        if (!x.exists) return x;
        const Tile tl = tiles[tile];
        x.d = descs + tl.slot;
        x.t = x.d->t + r;
        x.row = tl.row0 + warp * GPW + grp;
        x.valid = x.t < x.d->K && x.row < x.d->n;
        if (x.valid) {
            x.k0 = __ldg(x.d->row_ptr + x.row);
            x.k1 = __ldg(x.d->row_ptr + x.row + 1);
            if (x.d->hub_active && x.k1 - x.k0 > x.d->long_thresh) x.valid = false;   // long row: the long-row kernel's
        }
        return x;
    };

    // ask for the slices of item x this thread will read, into `stage`
    auto request = [&](const StreamItem &x, int stage) {
        const InstDesc *__restrict__ d = x.d;
        const int S_pad = d->S_pad;
        const size_t rbase = (size_t)x.row * S_pad;
        const T *Xc = reinterpret_cast<const T *>(d->X[x.t & 1]);
        const int npf = min(x.k1 - x.k0, NB);
#pragma unroll
        for (int v = 0; v < VPL; ++v) {
            const int off = (v * G + gl) * VEC;
            if (off < S_pad) {
                if (d->master) {
                    cp_async16(slot_ptr(stage, v, 0), d->master + rbase + off);
                    if (PW == 2) cp_async16(slot_ptr(stage, v, PW - 1), d->master + rbase + off + 4);
                } else {
                    cp_async16(slot_ptr(stage, v, 0), Xc + rbase + off);
                }
                cp_async16(slot_ptr(stage, v, PW), reinterpret_cast<const T *>(d->m) + rbase + off);
                cp_async16(slot_ptr(stage, v, PW + 1), reinterpret_cast<const T *>(d->v) + rbase + off);
            }
        }
        // neighbour indices are read G at a time by the group and broadcast
        for (int qb = 0; qb < npf; qb += G) {
            const int jl = qb + gl < npf ? __ldg(d->col + x.k0 + qb + gl) : 0;
            const int qn = min(G, npf - qb);
            for (int q = 0; q < qn; ++q) {
                const int j = __shfl_sync(gmask, jl, q, G);
#pragma unroll
                for (int v = 0; v < VPL; ++v) {
                    const int off = (v * G + gl) * VEC;
                    if (off < S_pad) cp_async16(slot_ptr(stage, v, PW + 2 + qb + q), Xc + (size_t)j * S_pad + off);
                }
            }
        }
    };

    StreamItem cur = fetch(0);
    if (cur.valid) request(cur, 0);
    cp_async_commit();
    for (int it = 0; cur.exists; ++it) {
        const int stage = it & 1;
        StreamItem nxt = fetch(it + 1);
        if (nxt.valid) request(nxt, stage ^ 1);
        cp_async_commit();
        cp_async_wait_1();   // everything but the newest group has landed: cur's slices
        if (cur.valid) {
            const InstDesc *__restrict__ d = cur.d;
            const StepCtx c = make_ctx(d, cur.t, r);
            OwnRow<T, G, VPL> own;
            float Y[VPL][VEC];
            float dsum = 0.0f;
            const int deg = cur.k1 - cur.k0;
            const int npf = min(deg, NB);
            const int32_t *__restrict__ wp = d->w;
#pragma unroll
            for (int v = 0; v < VPL; ++v) {
                const int off = (v * G + gl) * VEC;
#pragma unroll
                for (int e = 0; e < VEC; ++e) { Y[v][e] = 0.0f; own.P[v][e] = 0.0f; }
                own.M[v] = make_uint4(0, 0, 0, 0);
                own.V[v] = make_uint4(0, 0, 0, 0);
                if (off < c.S_pad) {
                    if (d->master) {
                        const uint4 a = *slot_ptr(stage, v, 0);
                        own.P[v][0] = __uint_as_float(a.x); own.P[v][1] = __uint_as_float(a.y);
                        own.P[v][2] = __uint_as_float(a.z); own.P[v][3] = __uint_as_float(a.w);
                        if (PW == 2) {
                            const uint4 b = *slot_ptr(stage, v, PW - 1);
                            own.P[v][4] = __uint_as_float(b.x); own.P[v][5] = __uint_as_float(b.y);
                            own.P[v][6] = __uint_as_float(b.z); own.P[v][7] = __uint_as_float(b.w);
                        }
                    } else {
                        VecT<T>::unpack(*slot_ptr(stage, v, 0), own.P[v]);
                    }
                    own.M[v] = *slot_ptr(stage, v, PW);
                    own.V[v] = *slot_ptr(stage, v, PW + 1);
                }
            }
            // prefetched neighbours, then the rest straight from global memory
            for (int q = 0; q < npf; ++q) {
                const float w = wp ? (float)__ldg(wp + cur.k0 + q) : 1.0f;
                dsum += w;
#pragma unroll
                for (int v = 0; v < VPL; ++v) {
                    const int off = (v * G + gl) * VEC;
                    if (off < c.S_pad) {
                        float x[VEC];
                        VecT<T>::unpack(*slot_ptr(stage, v, PW + 2 + q), x);
#pragma unroll
                        for (int e = 0; e < VEC; ++e) Y[v][e] = fmaf(w, x[e], Y[v][e]);
                    }
                }
            }
            if (deg > NB) {
                const T *__restrict__ Xc = reinterpret_cast<const T *>(d->X[c.t & 1]);
                for (int k = cur.k0 + NB; k < cur.k1; ++k) {
                    const int j = __ldg(d->col + k);
                    const float w = wp ? (float)__ldg(wp + k) : 1.0f;
                    dsum += w;
#pragma unroll
                    for (int v = 0; v < VPL; ++v) {
                        const int off = (v * G + gl) * VEC;
                        if (off < c.S_pad) {
                            float x[VEC];
                            VecT<T>::load_ro(Xc + (size_t)j * c.S_pad + off, x);
#pragma unroll
                            for (int e = 0; e < VEC; ++e) Y[v][e] = fmaf(w, x[e], Y[v][e]);
                        }
                    }
                }
            }
            update_row<T, G, VPL>(d, c, cur.row, gl, gmask, Y, dsum, own, status);
        }
        cur = nxt;
    }
}


// ---------------------------------------------------------------------------
// Long-row kernel. A row with more neighbours than the instance's long_thresh
// (a hub of a scale-free graph) would keep one lane group busy for the whole
// step while the rest of the grid idles, so its neighbour list is cut into
// segments of kSegLen consecutive CSR entries, each a separate work item: a
// lane group sums its segment (CSR order, as gather_row does) into an FP32
// partial row of the slot's seg_part, and the group that completes the row's
// last segment (an arrival counter per row; no group ever waits) adds the
// partials in segment order, Y = ((P_0 + P_1) + P_2) + ..., and runs the row's
// update. The order is fixed, so the result does not depend on which group
// finishes last, and every step kernel variant leaves these rows to this one.
// ---------------------------------------------------------------------------
template <typename T, int G, int VPL>
__global__ void __launch_bounds__(256) qqa_step_hub_kernel(const InstDesc *__restrict__ descs,
                                                           const Tile *__restrict__ items,
                                                           const int32_t *__restrict__ num_items_p,
                                                           RunStatus *__restrict__ status, int32_t r)
{
    constexpr int VEC = VecT<T>::N;
    const int lane = threadIdx.x & 31;
    const int gl = lane & (G - 1);
    const int grp = lane / G;
    const unsigned gmask = (G == 32) ? 0xffffffffu : (((1u << G) - 1u) << (grp * G));
    const int groups = (int)(blockDim.x / G);
    const int num_items = *num_items_p;
    const int stride = gridDim.x * groups;

    for (int it = blockIdx.x * groups + (int)(threadIdx.x / G); it < num_items; it += stride) {   // group-uniform
        const Tile itm = items[it];
        const InstDesc *__restrict__ d = descs + itm.slot;
        const int t = d->t + r;
        if (t >= d->K) continue;
        const int seg = itm.row0;
        const int j = __ldg(d->seg_row + seg);
        const int s0 = __ldg(d->seg_ptr + j), s1 = __ldg(d->seg_ptr + j + 1);
        const int row = __ldg(d->long_rows + j);
        const int rk0 = __ldg(d->row_ptr + row), rk1 = __ldg(d->row_ptr + row + 1);
        const int S_pad = d->S_pad;
        const T *__restrict__ Xc = reinterpret_cast<const T *>(d->X[t & 1]);
        RowIdx x{0, 0, 0, 0.0f};
        x.k0 = rk0 + (seg - s0) * kSegLen;
        x.k1 = min(x.k0 + kSegLen, rk1);
        if (x.k0 + gl < x.k1) {
            x.jl = __ldg(d->col + x.k0 + gl);
            x.wl = d->w ? (float)__ldg(d->w + x.k0 + gl) : 1.0f;
        }
        float Y[VPL][VEC];
#pragma unroll
        for (int v = 0; v < VPL; ++v)
#pragma unroll
            for (int e = 0; e < VEC; ++e) Y[v][e] = 0.0f;
        float dseg = 0.0f;
        gather_row<T, G, VPL>(d, Xc, x, S_pad, gl, gmask, Y, dseg);
        if (!seg_arrive<T, G, VPL>(d, seg, j, s0, s1, gl, gmask, Y)) continue;   // not the row's last segment
        const float dsum = row_weight_sum<G>(d, rk0, rk1, gl, gmask);
        const StepCtx c = make_ctx(d, t, r);
        OwnRow<T, G, VPL> own;
        load_own<T, G, VPL>(d, c, row, gl, own);
        update_row<T, G, VPL>(d, c, row, gl, gmask, Y, dsum, own, status);
    }
}

// ---------------------------------------------------------------------------
// One replica per node (S = 1, the paper's setting for random regular graphs):
// the state is one value per node (p[n] in FP32, or BF16 X with the FP32
// master; no padding lanes). A warp owns 32 consecutive rows. For the sparse
// product, groups of L lanes take one row each, L consecutive CSR entries per
// load (coalesced index loads); lane gl sums the entries k = k0 + gl (mod L)
// in CSR order, then the group adds its lanes by a fixed xor tree. Lane j then
// runs the update of row r0 + j (coalesced state accesses): with one replica
// the communication term of Eq. 10 is zero (p equals its own mean), the rest
// is the epilogue of the vector kernels for one element.
// ---------------------------------------------------------------------------
template <typename T>
__device__ __forceinline__ float load_scalar(const T *p);
template <>
__device__ __forceinline__ float load_scalar<float>(const float *p) { return __ldg(p); }
template <>
__device__ __forceinline__ float load_scalar<__nv_bfloat16>(const __nv_bfloat16 *p)
{
    const unsigned short u = __ldg(reinterpret_cast<const unsigned short *>(p));
    return __uint_as_float((uint32_t)u << 16);
}

template <typename T, int L>
__global__ void __launch_bounds__(256) qqa_step_scalar_kernel(const InstDesc *__restrict__ descs,
                                                              const Tile *__restrict__ tiles,
                                                              const int32_t *__restrict__ num_tiles_p,
                                                              RunStatus *__restrict__ status, int32_t r)
{
    constexpr int RPI = 32 / L;   // rows summed at once per warp (one per lane group)
    const int lane = threadIdx.x & 31;
    const int warp = threadIdx.x >> 5;
    const int gl = lane & (L - 1);
    const int grp = lane / L;
    const unsigned gmask = (L == 32) ? 0xffffffffu : (((1u << L) - 1u) << (grp * L));
    const int num_tiles = *num_tiles_p;

    for (int tile = blockIdx.x; tile < num_tiles; tile += gridDim.x) {
        const Tile tl = tiles[tile];
        const InstDesc *__restrict__ d = descs + tl.slot;
        const int t = d->t + r;
        if (t >= d->K) continue;   // block-uniform
        const int n = d->n;
        const int r0 = tl.row0 + warp * 32;
        if (r0 >= n) continue;     // warp-uniform
        const int row = r0 + lane;
        const bool live = row < n;
        // this lane's row: bounds, then its own state (in flight during the gather)
        const int kb = live ? __ldg(d->row_ptr + row) : 0;
        const int ke = live ? __ldg(d->row_ptr + row + 1) : 0;
        const T *__restrict__ Xc = reinterpret_cast<const T *>(d->X[t & 1]);
        float P = 0.0f, M = 0.0f, V = 0.0f;
        if (live) {
            P = d->master ? d->master[row] : load_scalar<T>(Xc + row);
            if (sizeof(T) == 4) {
                M = reinterpret_cast<const float *>(d->m)[row];
                V = reinterpret_cast<const float *>(d->v)[row];
            } else {
                M = load_scalar<__nv_bfloat16>(reinterpret_cast<const __nv_bfloat16 *>(d->m) + row);
                V = load_scalar<__nv_bfloat16>(reinterpret_cast<const __nv_bfloat16 *>(d->v) + row);
            }
        }
        const int32_t *__restrict__ colp = d->col;
        const int32_t *__restrict__ wp = d->w;
        float Ymine = 0.0f, Dmine = 0.0f;
#pragma unroll 1
        for (int it = 0; it < L; ++it) {
            const int src = it * RPI + grp;   // the warp's row this group sums now
            const int k0 = __shfl_sync(0xffffffffu, kb, src);
            const int k1 = __shfl_sync(0xffffffffu, ke, src);
            float y = 0.0f, ds = 0.0f;
#pragma unroll 4
            for (int k = k0 + gl; k < k1; k += L) {
                const int jn = __ldg(colp + k);
                const float wv = wp ? (float)__ldg(wp + k) : 1.0f;
                y = fmaf(wv, load_scalar<T>(Xc + jn), y);
                ds += wv;
            }
            y = group_sum<L>(y, gmask);
            ds = group_sum<L>(ds, gmask);
            // lane it * RPI + g takes the sum of group g
            const float yv = __shfl_sync(0xffffffffu, y, (lane % RPI) * L);
            const float dv = __shfl_sync(0xffffffffu, ds, (lane % RPI) * L);
            if (lane / RPI == it) {
                Ymine = yv;
                Dmine = dv;
            }
        }
        if (!live) continue;
        const StepCtx c = make_ctx(d, t, r);
        float g;
        if (c.kind == kMaxClique) g = fmaf(c.lambda, (c.cs_cur[0] - 0.5f) - Ymine, -1.0f);   // Eq. 24
        else if (c.kind == kMaxCut) g = fmaf(2.0f, Ymine, -Dmine);                            // Eq. 26
        else g = fmaf(c.lambda, Ymine, -1.0f);                                                // Eq. 22
        {   // annealed entropy term gamma_t (-2a) (2p - 1)^(a - 1) (Eq. 7)
            const float u = fmaf(2.0f, P, -1.0f);
            const float u2 = u * u;
            float upow = u;
            if (c.half_pow == 1) upow = u * u2;
            else
                for (int k = 0; k < c.half_pow; ++k) upow *= u2;
            g = fmaf(c.ent_coef, upow, g);
        }
        if (c.grad_dbg) c.grad_dbg[row] = g;
        // the Gaussian of replica 0: first Box-Muller value of node row's quad 0 (noise stream, step t)
        const U4 rq = philox10(U4{(uint32_t)row, 0u, (uint32_t)c.t, 1u}, d->seed_lo, d->seed_hi);
        float xi0, xi1;
        box_muller(rq.x, rq.y, xi0, xi1);
        const float mn = fmaf(c.b1, M, (1.0f - c.b1) * g);
        const float vn = fmaf(c.b2, V, (1.0f - c.b2) * (g * g));
        const float denom = fmaf(sqrt_nonneg(vn), c.inv_sqrt_bc2, c.adam_eps);
        float q = P * c.decay;
        q = fmaf(-c.step_size, mn * rcp_ftz(denom), q);
        const float pn = __saturatef(fmaf(c.noise_scale, xi0, q));
        if (!(vn <= 3.0e38f)) atomicAdd(&status->nonfinite, 1ULL);
        T *Xn = reinterpret_cast<T *>(d->X[(t + 1) & 1]);
        if (sizeof(T) == 4) {
            reinterpret_cast<float *>(Xn)[row] = pn;
            reinterpret_cast<float *>(d->m)[row] = mn;
            reinterpret_cast<float *>(d->v)[row] = vn;
        } else {
            d->master[row] = pn;
            reinterpret_cast<__nv_bfloat16 *>(Xn)[row] = __float2bfloat16_rn(pn);
            reinterpret_cast<__nv_bfloat16 *>(d->m)[row] = __float2bfloat16_rn(mn);
            reinterpret_cast<__nv_bfloat16 *>(d->v)[row] = __float2bfloat16_rn(vn);
        }
    }
}

}  // namespace qqa
