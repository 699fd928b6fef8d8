// color.cu -- categorical PQQA for graph colouring (App. B, App. C.4, App. D.1).
//
// State of one instance: W[i][k][s] in [0,1] for node i < n, colour k < K and
// replica s < S, with the AdamW moments m, v in the same layout, and the
// categorical relaxation sigma = W / sum_k W (Clamp-normalise, App. C.4; the
// clamp is the identity because every update ends with the projection to
// [0,1]). Rows of one (i, k) are S_pad = S rounded up to 32 floats long, so a
// warp reads 128 contiguous bytes of one colour plane.
//
// One step is the neighbour sums and the update:
//   neighbour sums  Y = A sigma, the relaxed-conflict sums, one of
//                   - color_planes_kernel + color_gather_tc_kernel: dense
//                     graphs (>= 5% of node pairs are edges) of 112 to 4096
//                     nodes, on the tensor cores (tcgen05);
//                   - color_gather_kernel: graphs of up to 1600 nodes, a
//                     sparse product over the columns (k, s) of sigma staged
//                     in shared memory;
//                   - larger graphs: gathered from global memory inside the
//                     update kernel;
//   color_update_kernel  one block per (node, 128 replicas), warp k = colour k,
//                        four replicas per lane:
//     statistics  mean and STD_eps of sigma_ik over the replicas, from the
//                 partial sums the previous step left
//     gradient    g_ik = Y_ik                                           relaxed conflicts
//                      + gamma_t (-c_K a K) (K sigma_ik - 1)^(a-1)      entropy s_K (App. B)
//                      - alpha (sigma_ik - mean_ik) / STD_ik            communication (Eq. 10)
//                 dR/dW_ik = (g_ik - sum_k' sigma_ik' g_ik') / sum_k W_ik   (Clamp-normalise chain rule)
//     update      AdamW with decoupled decay, + sqrt(2 lr T) xi, projection to [0,1]
//     relaxation  sigma' = W' / sum_k W' (a zero row: 1/K), into the other buffer,
//                 with the row sums sum_k W' for the next chain rule and the
//                 partial replica sums of sigma' for the next statistics
// sigma is double-buffered: a step reads sigma^t of the neighbours and writes
// sigma^{t+1} of its own node, so every block sees one consistent state.
//
// Rounding (color_argmax_kernel, color_conflict_kernel): x_is = argmax_k W_iks
// (equal to argmax sigma, the row sum is a positive common factor; ties go to
// the lowest colour, a zero row gives colour 0), then the conflicts
// sum_{edges i<j} [x_is = x_js] of every replica.
#include <algorithm>
#include <cmath>
#include <cstdarg>
#include <cstdio>
#include <cstring>
#include <new>
#include <type_traits>
#include <vector>

#include <cuda.h>
#include <cuda_fp16.h>

#include "../../include/qqa.h"
#include "qqa_internal.cuh"

namespace qqa {
int encode_tmap_f16_2d(void *map_out, const void *base, uint64_t inner, uint64_t outer, uint64_t row_bytes,
                       uint32_t box_inner, uint32_t box_outer);
int set_error(int code, const char *msg);
int check_unit_graph(int32_t n, const int32_t *rp, const int32_t *col);
void add_launches(unsigned long long k);
}  // namespace qqa

using namespace qqa;

namespace {


int cfail(int code, const char *fmt, ...)
{
    char buf[1024];
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(buf, sizeof buf, fmt, ap);
    va_end(ap);
    return set_error(code, buf);
}

#define COLOR_CK(call)                                                                             \
    do {                                                                                           \
        cudaError_t e_ = (call);                                                                   \
        if (e_ != cudaSuccess) return cfail(QQA_ECUDA, "%s: %s", #call, cudaGetErrorString(e_));   \
    } while (0)

// Arguments of one step. The step index is t = *t_dev + r: the device counter
// t_dev advances after every chunk of steps (so one captured CUDA graph serves
// every chunk of the same length) and r is the step's offset in its chunk.
// sched[t] = (gamma_t (-c_K a K), lr / (1 - b1^(t+1)), 1 / sqrt(1 - b2^(t+1)))
// is computed on the host in double and rounded once.
struct ColorStepArgs {
    int32_t n, K, S, S_pad, half_pow, r;
    const int32_t *t_dev;
    const float4 *sched;
    float decay;          // 1 - lr * weight_decay
    float b1, b2, adam_eps, alpha, comm_eps, noise_scale;
    uint32_t seed_lo, seed_hi;
};

// Replica statistics of sigma for the communication term (Eq. 10) are carried
// from step to step as per-chunk partial sums: for every (node i, colour k)
// and chunk c of 128 replicas, part[c] = (sum d, sum d^2) with d = sigma - h
// and the shift h = the mean of the previous step's sigma, so the one-pass
// variance sum d^2 / S - (sum d / S)^2 has no cancellation to speak of. The
// update kernel of a step combines the partials of its sigma and writes those
// of the next sigma; both are double-buffered by step parity.
constexpr int kMaxChunks = 8;   // chunks of 128 replicas (S <= 1024)

__device__ __forceinline__ float warp_sum(float x)
{
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) x += __shfl_xor_sync(0xffffffffu, x, o);
    return x;
}

// Partials of the sigma in buffer `sig` (a state set from the host, or the
// initial draw), one warp per (node, colour) row: the mean first (two passes),
// then the partials of every chunk about it.
__global__ void __launch_bounds__(256) color_stats_init_kernel(int32_t rows, int32_t S, int32_t S_pad,
                                                               const float *__restrict__ sig,
                                                               float2 *__restrict__ part, float *__restrict__ shift)
{
    const int r = (int)((blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5);
    const int lane = threadIdx.x & 31;
    if (r >= rows) return;
    const float *row = sig + (size_t)r * S_pad;
    float acc = 0.0f;
    for (int s = lane; s < S; s += 32) acc += row[s];
    const float mean = warp_sum(acc) / (float)S;
    const int chunks = (S_pad / 4 + 31) / 32;
    for (int c = 0; c < chunks; ++c) {
        float sd = 0.0f, sd2 = 0.0f;
        for (int e = 0; e < 4; ++e) {
            const int s = 128 * c + 4 * lane + e;
            if (s < S) {
                const float d = row[s] - mean;
                sd += d;
                sd2 = fmaf(d, d, sd2);
            }
        }
        sd = warp_sum(sd);
        sd2 = warp_sum(sd2);
        if (lane == 0) part[(size_t)r * kMaxChunks + c] = make_float2(sd, sd2);
    }
    if (lane == 0) shift[r] = mean;
}

__device__ __forceinline__ float4 ld4(const float *p) { return *reinterpret_cast<const float4 *>(p); }
__device__ __forceinline__ void st4(float *p, const float (&v)[4])
{
    *reinterpret_cast<float4 *>(p) = make_float4(v[0], v[1], v[2], v[3]);
}

// The step of node i = blockIdx.x / chunks for replica quads q = 32 c + lane,
// c = blockIdx.x % chunks: warp k of the block (K warps) owns colour k, so
// every access is a coalesced 16-byte-per-lane row of one (i, k) plane. The
// sums over colours (sum_k sigma_k g_k of the chain rule, sum_k W'_k of the
// next relaxation) meet in shared memory. With alpha != 0 the replica
// statistics of this step come from the partials (part, shift) of its parity,
// and the block writes those of the next sigma for its chunk; rsum[i][s]
// holds sum_k W of this step on entry and of the next on exit. Ygat is NULL
// for graphs too large for color_gather_kernel: the neighbour sums are then
// gathered here.
template <int MAXT>
__global__ void __launch_bounds__(MAXT)
color_update_kernel(ColorStepArgs a, int32_t chunks, const int32_t *__restrict__ rp, const int32_t *__restrict__ col,
                    float2 *__restrict__ part, float *__restrict__ shift, const float *__restrict__ Ygat,
                    float *__restrict__ sig0,
                    float *__restrict__ sig1, float *__restrict__ W, float *__restrict__ M,
                    float *__restrict__ V, float *__restrict__ rsum, float *__restrict__ grad_dbg,
                    unsigned long long *__restrict__ nonfinite)
{
    const int t = *a.t_dev + a.r;
    const float4 sc = a.sched[t];   // (entropy coefficient, step size, 1 / sqrt(bc2))
    const float *__restrict__ sig_cur = (t & 1) ? sig1 : sig0;
    float *__restrict__ sig_next = (t & 1) ? sig0 : sig1;
    __shared__ float4 xk[32][32];   // [colour][lane]: sigma_k g_k, then W'_k
    const int K = a.K;
    const int k = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int i = (int)(blockIdx.x / (unsigned)chunks);
    const int chunk = (int)(blockIdx.x % (unsigned)chunks);
    const int q = chunk * 32 + lane, s0 = 4 * q;
    const bool live = s0 < a.S;
    const size_t plane = (size_t)a.S_pad, node = (size_t)K * plane;
    const size_t idx = (size_t)i * node + (size_t)k * plane + s0;
    const float fK = (float)K;
    const bool comm = a.alpha != 0.0f;
    const size_t ik = (size_t)i * K + k, nk = (size_t)a.n * K;
    // mean and -alpha / STD of sigma_ik over the replicas (Eq. 10), from the partials
    float mean = 0.0f, coef = 0.0f;
    if (comm && k < K) {
        const float2 *__restrict__ pc = part + (size_t)(t & 1) * nk * kMaxChunks + ik * kMaxChunks;
        float sd = 0.0f, sd2 = 0.0f;
        for (int c = 0; c < chunks; ++c) {
            const float2 pv = pc[c];
            sd += pv.x;
            sd2 += pv.y;
        }
        const float inv_S = 1.0f / (float)a.S;
        const float md = sd * inv_S;
        mean = shift[(size_t)(t & 1) * nk + ik] + md;
        const float var = fmaxf(fmaf(sd2, inv_S, -md * md), 0.0f);
        coef = -a.alpha / sqrtf(var + a.comm_eps);
    }

    float g[4] = {0.0f, 0.0f, 0.0f, 0.0f}, sg[4] = {0.0f, 0.0f, 0.0f, 0.0f};
    // this lane's own state and noise, requested before the first barrier so
    // their latency overlaps the gradient and the exchange of the products
    float4 w4 = make_float4(0.0f, 0.0f, 0.0f, 0.0f), m4 = w4, v4 = w4, rs = w4;
    float xi[4] = {0.0f, 0.0f, 0.0f, 0.0f};
    if (live) {
        w4 = ld4(W + idx);
        m4 = ld4(M + idx);
        v4 = ld4(V + idx);
        rs = ld4(rsum + (size_t)i * plane + s0);
    }
    if (live) {
        // relaxed conflicts Y_ik
        if (Ygat) {
            const float4 y = ld4(Ygat + idx);
            g[0] = y.x, g[1] = y.y, g[2] = y.z, g[3] = y.w;
        } else {
            const float *__restrict__ base = sig_cur + (size_t)k * plane + s0;
            for (int e = rp[i]; e < rp[i + 1]; ++e) {
                const float4 y = ld4(base + (size_t)__ldg(col + e) * node);
                g[0] += y.x, g[1] += y.y, g[2] += y.z, g[3] += y.w;
            }
        }
        const float4 sv = ld4(sig_cur + idx);
        sg[0] = sv.x, sg[1] = sv.y, sg[2] = sv.z, sg[3] = sv.w;
        // dR/dsigma: + entropy s_K + communication
#pragma unroll
        for (int e = 0; e < 4; ++e) {
            const float u = fmaf(fK, sg[e], -1.0f);
            const float u2 = u * u;
            float upow = u;
            for (int h = 0; h < a.half_pow; ++h) upow *= u2;
            g[e] = fmaf(coef, sg[e] - mean, fmaf(sc.x, upow, g[e]));
        }
        if (a.noise_scale != 0.0f) gauss4(a.seed_lo, a.seed_hi, (uint32_t)(i * K + k), (uint32_t)q, (uint32_t)t, xi);
    }
    xk[k][lane] = make_float4(sg[0] * g[0], sg[1] * g[1], sg[2] * g[2], sg[3] * g[3]);
    __syncthreads();
    float dot[4] = {0.0f, 0.0f, 0.0f, 0.0f};
    for (int kk = 0; kk < K; ++kk) {
        const float4 d = xk[kk][lane];
        dot[0] += d.x, dot[1] += d.y, dot[2] += d.z, dot[3] += d.w;
    }
    float wn[4] = {0.0f, 0.0f, 0.0f, 0.0f};
    if (live) {
        // chain rule through W / sum W, AdamW, noise, projection
        const float rsv[4] = {rs.x, rs.y, rs.z, rs.w};
        const float w0[4] = {w4.x, w4.y, w4.z, w4.w}, m0[4] = {m4.x, m4.y, m4.z, m4.w},
                    v0[4] = {v4.x, v4.y, v4.z, v4.w};
        float gw[4], mn[4], vn[4];
        float vsum = 0.0f;
#pragma unroll
        for (int e = 0; e < 4; ++e) {
            gw[e] = rsv[e] > 0.0f ? (g[e] - dot[e]) / rsv[e] : 0.0f;
            mn[e] = fmaf(a.b1, m0[e], (1.0f - a.b1) * gw[e]);
            vn[e] = fmaf(a.b2, v0[e], (1.0f - a.b2) * (gw[e] * gw[e]));
            const float denom = fmaf(sqrtf(vn[e]), sc.z, a.adam_eps);
            const float qv = fmaf(-sc.y, mn[e] / denom, w0[e] * a.decay);
            wn[e] = __saturatef(fmaf(a.noise_scale, xi[e], qv));
            vsum += vn[e];
        }
        if (grad_dbg) st4(grad_dbg + idx, gw);
        st4(M + idx, mn);
        st4(V + idx, vn);
        st4(W + idx, wn);
        if (!(vsum <= 3.0e38f)) atomicAdd(nonfinite, 1ULL);
    }
    __syncthreads();   // every warp has read the products
    xk[k][lane] = make_float4(wn[0], wn[1], wn[2], wn[3]);
    __syncthreads();
    float ns[4] = {0.0f, 0.0f, 0.0f, 0.0f};
    for (int kk = 0; kk < K; ++kk) {
        const float4 d = xk[kk][lane];
        ns[0] += d.x, ns[1] += d.y, ns[2] += d.z, ns[3] += d.w;
    }
    float sd = 0.0f, sd2 = 0.0f;
    if (live) {
        // sigma' = W' / sum_k W' (1/K for a zero row), and the row sums
        float sp[4];
#pragma unroll
        for (int e = 0; e < 4; ++e) sp[e] = ns[e] > 0.0f ? wn[e] * (1.0f / ns[e]) : 1.0f / fK;
        st4(sig_next + idx, sp);
        if (k == 0) st4(rsum + (size_t)i * plane + s0, ns);
#pragma unroll
        for (int e = 0; e < 4; ++e)
            if (s0 + e < a.S) {
                const float d = sp[e] - mean;   // about this step's mean, the next step's shift
                sd += d;
                sd2 = fmaf(d, d, sd2);
            }
    }
    if (comm) {   // partials of the next sigma for this chunk (whole warps)
        sd = warp_sum(sd);
        sd2 = warp_sum(sd2);
        if (lane == 0) {
            const int tn = (t + 1) & 1;
            part[(size_t)tn * nk * kMaxChunks + ik * kMaxChunks + chunk] = make_float2(sd, sd2);
            if (chunk == 0) shift[(size_t)tn * nk + ik] = mean;
        }
    }
}

// Neighbour sums Y = A sigma of the relaxed conflicts for graphs whose slab
// fits in shared memory. sigma is read as a matrix [n][C], C = K * S_pad (row
// j = all colours and replicas of node j). Block b stages the 32 VEC columns
// [32 VEC c, 32 VEC (c + 1)) of every row, c = b / parts (n * 128 VEC bytes),
// then each warp sums, for its rows i of part b % parts, the staged rows of
// i's neighbours, VEC columns per lane. Neighbour indices are read 32 at a
// time and broadcast by shuffles.
template <int VEC>
__global__ void __launch_bounds__(256) color_gather_kernel(int32_t n, int64_t C, int32_t parts,
                                                           const int32_t *__restrict__ rp,
                                                           const int32_t *__restrict__ col,
                                                           const float *__restrict__ sig0,
                                                           const float *__restrict__ sig1,
                                                           const int32_t *__restrict__ t_dev, int32_t step_off,
                                                           float *__restrict__ Y)
{
    const float *__restrict__ sig = ((*t_dev + step_off) & 1) ? sig1 : sig0;
    using V = typename std::conditional<VEC == 4, float4, typename std::conditional<VEC == 2, float2, float>::type>::type;
    extern __shared__ __align__(16) unsigned char slab_raw[];
    V *slab = reinterpret_cast<V *>(slab_raw);   // [n][32]
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
    const int chunk = (int)(blockIdx.x / (unsigned)parts), part = (int)(blockIdx.x % (unsigned)parts);
    const int64_t c0 = ((int64_t)chunk * 32 + lane) * VEC;
#pragma unroll 4
    for (int j = warp; j < n; j += nw) slab[j * 32 + lane] = *reinterpret_cast<const V *>(sig + (int64_t)j * C + c0);
    __syncthreads();
    const int rows = (n + parts - 1) / parts;
    const int r1 = min(n, (part + 1) * rows);
    for (int i = part * rows + warp; i < r1; i += nw) {
        const int e0 = rp[i], e1 = rp[i + 1];
        V y0, y1;
        if constexpr (VEC == 4) {
            y0 = make_float4(0.0f, 0.0f, 0.0f, 0.0f);
        } else if constexpr (VEC == 2) {
            y0 = make_float2(0.0f, 0.0f);
        } else {
            y0 = 0.0f;
        }
        y1 = y0;
        for (int eb = e0; eb < e1; eb += 32) {
            const int cnt = min(32, e1 - eb);
            const int mine = lane < cnt ? col[eb + lane] : 0;
            int qq = 0;
            for (; qq + 1 < cnt; qq += 2) {
                const V a0 = slab[__shfl_sync(0xffffffffu, mine, qq) * 32 + lane];
                const V a1 = slab[__shfl_sync(0xffffffffu, mine, qq + 1) * 32 + lane];
                if constexpr (VEC == 4) {
                    y0.x += a0.x, y0.y += a0.y, y0.z += a0.z, y0.w += a0.w;
                    y1.x += a1.x, y1.y += a1.y, y1.z += a1.z, y1.w += a1.w;
                } else if constexpr (VEC == 2) {
                    y0.x += a0.x, y0.y += a0.y;
                    y1.x += a1.x, y1.y += a1.y;
                } else {
                    y0 += a0;
                    y1 += a1;
                }
            }
            if (qq < cnt) {
                const V a0 = slab[__shfl_sync(0xffffffffu, mine, qq) * 32 + lane];
                if constexpr (VEC == 4) {
                    y0.x += a0.x, y0.y += a0.y, y0.z += a0.z, y0.w += a0.w;
                } else if constexpr (VEC == 2) {
                    y0.x += a0.x, y0.y += a0.y;
                } else {
                    y0 += a0;
                }
            }
        }
        if constexpr (VEC == 4)
            *reinterpret_cast<float4 *>(Y + (int64_t)i * C + c0) =
                make_float4(y0.x + y1.x, y0.y + y1.y, y0.z + y1.z, y0.w + y1.w);
        else if constexpr (VEC == 2)
            *reinterpret_cast<float2 *>(Y + (int64_t)i * C + c0) = make_float2(y0.x + y1.x, y0.y + y1.y);
        else
            Y[(int64_t)i * C + c0] = y0 + y1;
    }
}

// ---------------------------------------------------------------------------
// Neighbour sums on the tensor cores, for dense graphs of up to 4096 nodes:
// Y = A sigma with A the 0/1 adjacency in fp16 [n_pad][n_pad] (exact) and
// sigma in two fp16 planes stored transposed, [C][n_pad] (C = K * S_pad):
// hi = fp16(sigma) and lo = fp16((sigma - hi) * 2^12). hi + lo 2^-12 carries
// about 22 significant bits; the scale keeps lo a normal fp16 number for every
// sigma in [0, 1]. The two products accumulate in separate FP32 tensor-memory
// accumulators (every product is exact) and Y = D_hi + 2^-12 D_lo.
// ---------------------------------------------------------------------------
constexpr int kTcMinNodes = 112, kTcMaxNodes = 4096;
constexpr double kTcMinDensity = 0.05;   // nnz / n^2 below which the dense product wastes the tensor cores

// sigma [n][C] -> hi, lo planes [C][n_pad], through a 64 x 32 shared tile
__global__ void __launch_bounds__(256) color_planes_kernel(int32_t n, int32_t n_pad, int32_t C,
                                                           const float *__restrict__ sig0,
                                                           const float *__restrict__ sig1,
                                                           const int32_t *__restrict__ t_dev, int32_t step_off,
                                                           __half *__restrict__ hi, __half *__restrict__ lo)
{
    __shared__ float tile[64][33];
    const float *__restrict__ sig = ((*t_dev + step_off) & 1) ? sig1 : sig0;
    const int i0 = blockIdx.x * 32, c0 = blockIdx.y * 64;
    for (int e = threadIdx.x; e < 32 * 64; e += blockDim.x) {
        const int r = e >> 6, cc = e & 63;
        const int i = i0 + r, c = c0 + cc;
        tile[cc][r] = (i < n && c < C) ? sig[(size_t)i * C + c] : 0.0f;
    }
    __syncthreads();
    for (int e = threadIdx.x; e < 32 * 64; e += blockDim.x) {
        const int cc = e >> 5, r = e & 31;
        const int i = i0 + r, c = c0 + cc;
        if (i < n && c < C) {
            const float x = tile[cc][r];
            const __half h = __float2half_rn(x);
            hi[(size_t)c * n_pad + i] = h;
            lo[(size_t)c * n_pad + i] = __float2half_rn((x - __half2float(h)) * 4096.0f);
        }
    }
}

__device__ __forceinline__ uint32_t smem_addr(const void *p) { return (uint32_t)__cvta_generic_to_shared(p); }

__device__ __forceinline__ uint64_t tc_desc_sw128(uint32_t saddr)
{
    // K-major operand with 128-byte swizzle: start address >> 4, leading byte
    // offset 1 (unused by this layout), stride byte offset 1024 >> 4 (eight
    // 128-byte rows), descriptor version 1, layout 2 (128-byte swizzle)
    return (uint64_t)((saddr >> 4) & 0x3FFF) | ((uint64_t)1 << 16) | ((uint64_t)64 << 32) | ((uint64_t)1 << 46) |
           ((uint64_t)2 << 61);
}

__device__ __forceinline__ void tc_tma_load_2d(uint32_t dst, const void *tmap, int x, int y, uint32_t mbar)
{
    asm volatile(
        "cp.async.bulk.tensor.2d.shared::cluster.global.tile.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3}], [%4];" ::"r"(
            dst),
        "l"(tmap), "r"(x), "r"(y), "r"(mbar)
        : "memory");
}

__device__ __forceinline__ void tc_mma_f16(uint32_t tmem_d, uint64_t a, uint64_t b, uint32_t idesc, uint32_t accumulate)
{
    asm volatile("{\n\t.reg .pred p;\n\tsetp.ne.b32 p, %4, 0;\n\t"
                 "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n\t}" ::"r"(tmem_d),
                 "l"(a), "l"(b), "r"(idesc), "r"(accumulate)
                 : "memory");
}

__device__ __forceinline__ void tc_commit(uint32_t mbar)
{
    asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(mbar) : "memory");
}

__device__ __forceinline__ void tc_ld16(uint32_t taddr, uint32_t (&r)[16])
{
    asm volatile("tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15}, [%16];"
                 : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]),
                   "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15])
                 : "r"(taddr));
    asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
}

// Wait for phase `parity` of an mbarrier, for about a second at most.
__device__ __forceinline__ bool tc_wait(uint32_t mbar, uint32_t parity)
{
    const long long start = clock64();
    while (true) {
        uint32_t ok;
        asm volatile("{\n\t.reg .pred p;\n\tmbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\tselp.u32 %0, 1, 0, p;\n\t}"
                     : "=r"(ok)
                     : "r"(mbar), "r"(parity)
                     : "memory");
        if (ok) return true;
        if (clock64() - start > (1LL << 31)) return false;
    }
}

constexpr int kTcStages = 2;
constexpr int kTcThreads = 160;   // 4 epilogue warps (TMEM lanes 0..127) + 1 control warp

__host__ __device__ constexpr int tc_stage_bytes(int NT) { return 128 * 128 + 2 * NT * 128; }
__host__ __device__ constexpr int tc_smem_bytes(int NT) { return 1024 + kTcStages * tc_stage_bytes(NT) + 64; }

// One CTA per (128-row tile m, NT-column tile c): D_hi, D_lo = A[m rows] . {hi, lo}[c cols]^T
// over K = n_pad in 64-wide chunks (TMA, two stages, bounded waits), then
// Y[row][c0 + col] = D_hi + 2^-12 D_lo for the tile's rows below n.
// tmaps: A, hi, lo (device copies of CUtensorMap).
template <int NT>
__global__ void __launch_bounds__(kTcThreads, 1)
color_gather_tc_kernel(int32_t n, int32_t n_pad, int64_t C, const void *__restrict__ tmaps, float *__restrict__ Y,
                       unsigned long long *__restrict__ timeouts)
{
    constexpr int A_BYTES = 128 * 128, B_BYTES = NT * 128, STAGE = tc_stage_bytes(NT);
    extern __shared__ __align__(1024) unsigned char tc_raw[];
    unsigned char *base = (unsigned char *)(((uintptr_t)tc_raw + 1023) & ~(uintptr_t)1023);
    uint64_t *mb_full = reinterpret_cast<uint64_t *>(base + kTcStages * STAGE);
    uint64_t *mb_empty = mb_full + kTcStages;
    uint64_t *mb_acc = mb_empty + kTcStages;
    uint32_t *tmem_slot = reinterpret_cast<uint32_t *>(mb_acc + 1);
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int row0 = blockIdx.x * 128;
    const int c0 = blockIdx.y * NT;
    const int nK = n_pad / 64;

    if (threadIdx.x == 0) {
        for (int k = 0; k < kTcStages; ++k) {
            asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(smem_addr(mb_full + k)) : "memory");
            asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(smem_addr(mb_empty + k)) : "memory");
        }
        asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(smem_addr(mb_acc)) : "memory");
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    if (warp == 0) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_addr(tmem_slot)),
                     "n"(2 * NT)
                     : "memory");
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
    }
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncthreads();
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    const uint32_t tmem = *tmem_slot;

    bool ok = true;
    if (warp == 4) {
        if (lane == 0) {
            const CUtensorMap *tm = reinterpret_cast<const CUtensorMap *>(tmaps);
            const CUtensorMap *tmA = tm, *tmH = tm + 1, *tmL = tm + 2;
            asm volatile("fence.proxy.tensormap::generic.acquire.gpu [%0], 128;" ::"l"(tmA) : "memory");
            asm volatile("fence.proxy.tensormap::generic.acquire.gpu [%0], 128;" ::"l"(tmH) : "memory");
            asm volatile("fence.proxy.tensormap::generic.acquire.gpu [%0], 128;" ::"l"(tmL) : "memory");
            const uint32_t idesc = (1u << 4) | ((uint32_t)(NT >> 3) << 17) | ((uint32_t)(128 >> 4) << 24);
            auto fill = [&](int kc) {
                const int st = kc % kTcStages;
                if (kc >= kTcStages) ok = ok && tc_wait(smem_addr(mb_empty + st), ((kc / kTcStages) - 1) & 1);
                if (!ok) return;
                unsigned char *sp = base + st * STAGE;
                asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_addr(mb_full + st)),
                             "r"(STAGE)
                             : "memory");
                tc_tma_load_2d(smem_addr(sp), tmA, 64 * kc, row0, smem_addr(mb_full + st));
                tc_tma_load_2d(smem_addr(sp + A_BYTES), tmH, 64 * kc, c0, smem_addr(mb_full + st));
                tc_tma_load_2d(smem_addr(sp + A_BYTES + B_BYTES), tmL, 64 * kc, c0, smem_addr(mb_full + st));
            };
            for (int kc = 0; kc < kTcStages && kc < nK; ++kc) fill(kc);
            for (int kc = 0; kc < nK && ok; ++kc) {
                const int st = kc % kTcStages;
                ok = tc_wait(smem_addr(mb_full + st), (kc / kTcStages) & 1);
                if (!ok) break;
                asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
                const uint32_t sa = smem_addr(base + st * STAGE);
#pragma unroll
                for (int ks = 0; ks < 4; ++ks) {
                    const uint64_t ad = tc_desc_sw128(sa + ks * 32);
                    const uint64_t bh = tc_desc_sw128(sa + A_BYTES + ks * 32);
                    const uint64_t bl = tc_desc_sw128(sa + A_BYTES + B_BYTES + ks * 32);
                    const uint32_t acc = (kc > 0 || ks > 0) ? 1u : 0u;
                    tc_mma_f16(tmem, ad, bh, idesc, acc);
                    tc_mma_f16(tmem + NT, ad, bl, idesc, acc);
                }
                tc_commit(smem_addr(mb_empty + st));   // stage free once these MMAs are done
                if (kc + kTcStages < nK) fill(kc + kTcStages);
            }
            if (ok) tc_commit(smem_addr(mb_acc));
            else atomicAdd(timeouts, 1ULL);
        }
        __syncwarp();
    } else {
        // epilogue warps: TMEM lane = row of the tile
        const bool acc_ok = tc_wait(smem_addr(mb_acc), 0);
        asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
        if (!acc_ok) {
            if (threadIdx.x == 0) atomicAdd(timeouts, 1ULL);
        } else {
            const int row = row0 + 32 * warp + lane;
            float *__restrict__ yrow = Y + (size_t)row * C + c0;
#pragma unroll 1
            for (int c16 = 0; c16 < NT; c16 += 16) {
                uint32_t vh[16], vl[16];
                tc_ld16(tmem + ((uint32_t)(32 * warp) << 16) + (uint32_t)c16, vh);
                tc_ld16(tmem + ((uint32_t)(32 * warp) << 16) + (uint32_t)(NT + c16), vl);
                if (row < n) {
#pragma unroll
                    for (int e = 0; e < 16; e += 4)
                        *reinterpret_cast<float4 *>(yrow + c16 + e) =
                            make_float4(fmaf(__uint_as_float(vl[e]), 2.44140625e-4f, __uint_as_float(vh[e])),
                                        fmaf(__uint_as_float(vl[e + 1]), 2.44140625e-4f, __uint_as_float(vh[e + 1])),
                                        fmaf(__uint_as_float(vl[e + 2]), 2.44140625e-4f, __uint_as_float(vh[e + 2])),
                                        fmaf(__uint_as_float(vl[e + 3]), 2.44140625e-4f, __uint_as_float(vh[e + 3])));
                }
            }
        }
        asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    }
    __syncthreads();
    if (warp == 0) {
        asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "n"(2 * NT) : "memory");
    }
}

// The step counter of the device: advanced after each chunk, set from the host.
__global__ void color_advance_kernel(int32_t *t_dev, int32_t by) { *t_dev += by; }
__global__ void color_set_t_kernel(int32_t *t_dev, int32_t t) { *t_dev = t; }

// sigma = W / sum_k W for every (i, s) (1/K for a zero row), and the row sums.
__global__ void color_sigma_kernel(int32_t n, int32_t K, int32_t S, int32_t S_pad, const float *__restrict__ W,
                                   float *__restrict__ sig, float *__restrict__ rsum)
{
    const int64_t idx = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (idx >= (int64_t)n * S_pad) return;
    const int64_t i = idx / S_pad;
    const int s = (int)(idx % S_pad);
    if (s >= S) return;
    const float *w = W + i * K * S_pad + s;
    float sum = 0.0f;
    for (int k = 0; k < K; ++k) sum += w[(int64_t)k * S_pad];
    float *o = sig + i * K * S_pad + s;
    const float inv = sum > 0.0f ? 1.0f / sum : 0.0f;
    for (int k = 0; k < K; ++k) o[(int64_t)k * S_pad] = sum > 0.0f ? w[(int64_t)k * S_pad] * inv : 1.0f / (float)K;
    rsum[idx] = sum;
}

// W = U(0,1] of Philox block (i*K + k, s/4, 0, 0), element s mod 4 (the binary
// method's initial draw with row index i*K + k).
__global__ void color_init_kernel(int32_t n, int32_t K, int32_t S, int32_t S_pad, uint32_t lo, uint32_t hi,
                                  float *__restrict__ W)
{
    const int64_t idx = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (idx >= (int64_t)n * K * S_pad) return;
    const uint32_t row = (uint32_t)(idx / S_pad);
    const int s = (int)(idx % S_pad);
    if (s >= S) {
        W[idx] = 0.0f;
        return;
    }
    const U4 r = philox10(U4{row, (uint32_t)(s >> 2), 0u, 0u}, lo, hi);
    const uint32_t b = (s & 2) ? ((s & 1) ? r.w : r.z) : ((s & 1) ? r.y : r.x);
    W[idx] = bits_to_unit(b);
}

// x_is = argmax_k W_iks, ties to the lowest k.
__global__ void color_argmax_kernel(int32_t n, int32_t K, int32_t S, int32_t S_pad, const float *__restrict__ W,
                                    uint8_t *__restrict__ x)
{
    const int64_t idx = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (idx >= (int64_t)n * S_pad) return;
    const int64_t i = idx / S_pad;
    const int s = (int)(idx % S_pad);
    if (s >= S) return;
    const float *w = W + i * K * S_pad + s;
    int arg = 0;
    float best = w[0];
    for (int k = 1; k < K; ++k) {
        const float v = w[(int64_t)k * S_pad];
        if (v > best) {
            best = v;
            arg = k;
        }
    }
    x[idx] = (uint8_t)arg;
}

// conflicts[s] += #{ j in N(i), j > i : x_js = x_is }
__global__ void color_conflict_kernel(int32_t n, int32_t S, int32_t S_pad, const int32_t *__restrict__ rp,
                                      const int32_t *__restrict__ col, const uint8_t *__restrict__ x,
                                      unsigned long long *__restrict__ conflicts)
{
    const int64_t idx = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (idx >= (int64_t)n * S_pad) return;
    const int32_t i = (int32_t)(idx / S_pad);
    const int s = (int)(idx % S_pad);
    if (s >= S) return;
    const uint8_t xi = x[idx];
    unsigned int c = 0;
    for (int e = rp[i]; e < rp[i + 1]; ++e) {
        const int32_t j = col[e];
        if (j > i && x[(int64_t)j * S_pad + s] == xi) ++c;
    }
    if (c) atomicAdd(conflicts + s, (unsigned long long)c);
}

// Largest shared-memory slab of color_gather_kernel (n * 128 VEC bytes).
constexpr int kGatherSlabMax = 200 * 1024;

}  // namespace

struct qqa_color {
    int32_t n = 0, K = 0, S = 0, S_pad = 0, t = 0;
    int64_t nnz = 0;
    qqa_params prm{};
    double cK = 0.0;
    cudaStream_t st = nullptr;
    int sms = 0;
    int32_t *rp = nullptr, *col = nullptr;
    float *W = nullptr, *m = nullptr, *v = nullptr, *sig[2] = {nullptr, nullptr}, *grad = nullptr;
    float2 *part = nullptr;   // [2][n][K][kMaxChunks] partial replica sums of sigma
    float *shift = nullptr;   // [2][n][K] their shifts
    float *rsum = nullptr;    // sum_k W per (node, replica)
    float *Y = nullptr;       // neighbour sums when the graph fits color_gather_kernel's slab
    int gather_vec = 0;       // 4, 2 or 1: columns per lane of color_gather_kernel; 0: direct gather
    int tc_nt = 0;            // > 0: neighbour sums on the tensor cores, NT columns per CTA
    int n_pad = 0;            // n rounded up to 128 (tensor-core path)
    __half *A16 = nullptr, *hi = nullptr, *lo = nullptr;   // fp16 adjacency and sigma planes
    void *tmaps = nullptr;    // tensor maps of A16, hi, lo
    unsigned long long *timeouts = nullptr;
    int32_t *t_dev = nullptr; // step counter of the device
    float4 *sched = nullptr;  // per-step scalars, [steps]
    uint8_t *x = nullptr;
    unsigned long long *conf = nullptr, *nonfinite = nullptr;
    std::vector<void *> owned;
    cudaStream_t cap_stream = nullptr;     // private stream the step chunk is captured on
    cudaGraphExec_t chunk_exec = nullptr;  // kColorChunk steps and the counter advance
    int chunk_kernels = 0;                 // kernels per replay of chunk_exec

    size_t nks() const { return (size_t)n * (size_t)K * (size_t)S_pad; }
};

static void color_free(qqa_color *c)
{
    if (!c) return;
    if (c->st) cudaStreamSynchronize(c->st);
    else cudaDeviceSynchronize();
    if (c->chunk_exec) cudaGraphExecDestroy(c->chunk_exec);
    if (c->cap_stream) cudaStreamDestroy(c->cap_stream);
    for (void *p : c->owned) cudaFree(p);
    delete c;
}

template <typename T>
static T *color_alloc(qqa_color *c, size_t count)
{
    void *p = nullptr;
    if (cudaMalloc(&p, std::max<size_t>(count * sizeof(T), 16)) != cudaSuccess) {
        (void)cudaGetLastError();
        return nullptr;
    }
    c->owned.push_back(p);
    return (T *)p;
}

// sigma and the row sums of the current W into buffer `which`, and the
// partial replica sums of that sigma.
static int color_launch_sigma(qqa_color *c, int which)
{
    const int64_t total = (int64_t)c->n * c->S_pad;
    color_sigma_kernel<<<(unsigned)((total + 255) / 256), 256, 0, c->st>>>(c->n, c->K, c->S, c->S_pad, c->W,
                                                                        c->sig[which], c->rsum);
    const int rows = c->n * c->K;
    color_stats_init_kernel<<<(unsigned)((rows + 7) / 8), 256, 0, c->st>>>(
        rows, c->S, c->S_pad, c->sig[which], c->part + (size_t)which * rows * kMaxChunks, c->shift + (size_t)which * rows);
    COLOR_CK(cudaGetLastError());
    add_launches(2);
    return QQA_OK;
}

// Steps replayed per CUDA graph launch.
constexpr int kColorChunk = 32;

// Enqueue steps t .. t + L - 1 (t = the device counter) on stream st, then
// advance the counter by L. Returns the number of kernels enqueued, or a
// negative error code.
static int color_enqueue_chunk(qqa_color *c, int L, float *grad_dbg, cudaStream_t st)
{
    const qqa_params &p = c->prm;
    ColorStepArgs a{};
    a.n = c->n;
    a.K = c->K;
    a.S = c->S;
    a.S_pad = c->S_pad;
    a.half_pow = (p.a_ent - 2) / 2;
    a.t_dev = c->t_dev;
    a.sched = c->sched;
    a.decay = (float)(1.0 - (double)p.lr * (double)p.weight_decay);
    a.b1 = p.beta1;
    a.b2 = p.beta2;
    a.adam_eps = p.adam_eps;
    a.alpha = p.alpha_comm;
    a.comm_eps = p.comm_eps;
    a.noise_scale = (float)std::sqrt(2.0 * (double)p.lr * (double)p.temperature);
    a.seed_lo = (uint32_t)(p.seed & 0xffffffffu);
    a.seed_hi = (uint32_t)(p.seed >> 32);
    int kernels = 0;
    for (int r = 0; r < L; ++r) {
        a.r = r;
        const float *Ygat = nullptr;
        if (c->tc_nt) {
            const int C = c->K * c->S_pad;
            color_planes_kernel<<<dim3((unsigned)((c->n + 31) / 32), (unsigned)((C + 63) / 64)), 256, 0, st>>>(
                c->n, c->n_pad, C, c->sig[0], c->sig[1], c->t_dev, r, c->hi, c->lo);
            const dim3 grid((unsigned)(c->n_pad / 128), (unsigned)(C / c->tc_nt));
            if (c->tc_nt == 128)
                color_gather_tc_kernel<128><<<grid, kTcThreads, tc_smem_bytes(128), st>>>(c->n, c->n_pad, C, c->tmaps,
                                                                                        c->Y, c->timeouts);
            else
                color_gather_tc_kernel<64><<<grid, kTcThreads, tc_smem_bytes(64), st>>>(c->n, c->n_pad, C, c->tmaps,
                                                                                      c->Y, c->timeouts);
            kernels += 2;
            Ygat = c->Y;
        } else if (c->gather_vec) {
            const int vec = c->gather_vec;
            const int64_t C = (int64_t)c->K * c->S_pad;
            const int smem = c->n * 128 * vec;
            const int64_t chunks = C / (32 * vec);
            // split the rows so that the blocks fill the GPU in one wave
            const int64_t per_sm = std::max(1, std::min(8, (228 * 1024) / (smem + 1024)));
            const int64_t slots = per_sm * c->sms;
            const int parts = (int)std::max<int64_t>(1, std::min<int64_t>(slots / chunks, (c->n + 31) / 32));
            const unsigned grid = (unsigned)(chunks * parts);
            if (vec == 4)
                color_gather_kernel<4><<<grid, 256, smem, st>>>(c->n, C, parts, c->rp, c->col, c->sig[0], c->sig[1],
                                                                c->t_dev, r, c->Y);
            else if (vec == 2)
                color_gather_kernel<2><<<grid, 256, smem, st>>>(c->n, C, parts, c->rp, c->col, c->sig[0], c->sig[1],
                                                                c->t_dev, r, c->Y);
            else
                color_gather_kernel<1><<<grid, 256, smem, st>>>(c->n, C, parts, c->rp, c->col, c->sig[0], c->sig[1],
                                                                c->t_dev, r, c->Y);
            ++kernels;
            Ygat = c->Y;
        }
        const int chunks = (c->S_pad / 4 + 31) / 32;   // 32 quads of replicas per block
        auto update = c->K <= 16 ? color_update_kernel<512> : color_update_kernel<1024>;
        update<<<(unsigned)((int64_t)c->n * chunks), 32 * c->K, 0, st>>>(
            a, chunks, c->rp, c->col, c->part, c->shift, Ygat, c->sig[0], c->sig[1], c->W, c->m, c->v, c->rsum, grad_dbg,
            c->nonfinite);
        ++kernels;
    }
    color_advance_kernel<<<1, 1, 0, st>>>(c->t_dev, L);
    ++kernels;
    const cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return cfail(QQA_ECUDA, "colouring step launch: %s", cudaGetErrorString(e));
    return kernels;
}

// Run L steps: full chunks replay one captured graph (captured on first use
// on a private stream, launched on the handle's stream), the rest are
// launched directly.
static int color_run(qqa_color *c, int L)
{
    while (L > 0) {
        const int len = std::min(L, kColorChunk);
        if (len == kColorChunk) {
            if (!c->chunk_exec) {
                if (!c->cap_stream) COLOR_CK(cudaStreamCreateWithFlags(&c->cap_stream, cudaStreamNonBlocking));
                cudaGraph_t g = nullptr;
                COLOR_CK(cudaStreamBeginCapture(c->cap_stream, cudaStreamCaptureModeThreadLocal));
                const int k = color_enqueue_chunk(c, kColorChunk, nullptr, c->cap_stream);
                const cudaError_t e = cudaStreamEndCapture(c->cap_stream, &g);
                if (k < 0) {
                    if (g) cudaGraphDestroy(g);
                    return k;
                }
                if (e != cudaSuccess) return cfail(QQA_ECUDA, "colouring chunk capture: %s", cudaGetErrorString(e));
                const cudaError_t ei = cudaGraphInstantiate(&c->chunk_exec, g, 0);
                cudaGraphDestroy(g);
                if (ei != cudaSuccess) {
                    c->chunk_exec = nullptr;
                    return cfail(QQA_ECUDA, "colouring chunk instantiate: %s", cudaGetErrorString(ei));
                }
                c->chunk_kernels = k;
            }
            COLOR_CK(cudaGraphLaunch(c->chunk_exec, c->st));
            add_launches((unsigned long long)c->chunk_kernels);
        } else {
            const int k = color_enqueue_chunk(c, len, nullptr, c->st);
            if (k < 0) return k;
            add_launches((unsigned long long)k);
        }
        c->t += len;
        L -= len;
    }
    return QQA_OK;
}

extern "C" int qqa_color_create(int32_t n, const int32_t *row_ptr, const int32_t *col, int32_t K,
                                const qqa_params *prm, void *stream, qqa_color **out)
{
    if (!out) return cfail(QQA_EINVAL, "out is NULL");
    *out = nullptr;
    if (!prm) return cfail(QQA_EINVAL, "params is NULL");
    if (K < 2 || K > QQA_COLOR_MAX_K) return cfail(QQA_EINVAL, "K must be in [2, %d] (got %d)", QQA_COLOR_MAX_K, K);
    if (prm->S < 1 || prm->S > 1024) return cfail(QQA_EINVAL, "S must be in [1, 1024] (got %d)", prm->S);
    if (prm->steps < 1) return cfail(QQA_EINVAL, "steps must be >= 1 (got %d)", prm->steps);
    if (prm->a_ent < 2 || prm->a_ent > 8 || (prm->a_ent & 1))
        return cfail(QQA_EINVAL, "a_ent must be 2, 4, 6 or 8 (got %d)", prm->a_ent);
    if (prm->precision != QQA_FP32) return cfail(QQA_EINVAL, "colouring runs in FP32 only");
    if ((int64_t)n * K > 0x7fffffffLL) return cfail(QQA_EINVAL, "n * K exceeds the 32-bit counter row");
    int rc = check_unit_graph(n, row_ptr, col);
    if (rc != QQA_OK) return rc;

    qqa_color *c = new (std::nothrow) qqa_color();
    if (!c) return cfail(QQA_ENOMEM, "host allocation failed");
    c->n = n;
    c->K = K;
    c->S = prm->S;
    c->S_pad = (prm->S + 31) / 32 * 32;
    c->nnz = row_ptr[n];
    c->prm = *prm;
    c->st = (cudaStream_t)stream;
    {
        double pw = 1.0;
        for (int h = 0; h < prm->a_ent - 1; ++h) pw *= (double)(K - 1);
        c->cK = 1.0 / ((double)(K - 1) * (pw + 1.0));
    }
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || cudaDeviceGetAttribute(&c->sms, cudaDevAttrMultiProcessorCount, dev) !=
                                                  cudaSuccess) {
        (void)cudaGetLastError();
        delete c;
        return cfail(QQA_ECUDA, "no CUDA device");
    }
    const size_t nks = c->nks();
    c->rp = color_alloc<int32_t>(c, (size_t)n + 1);
    c->col = color_alloc<int32_t>(c, (size_t)std::max<int64_t>(c->nnz, 1));
    c->W = color_alloc<float>(c, nks);
    c->m = color_alloc<float>(c, nks);
    c->v = color_alloc<float>(c, nks);
    c->sig[0] = color_alloc<float>(c, nks);
    c->sig[1] = color_alloc<float>(c, nks);
    c->x = color_alloc<uint8_t>(c, (size_t)n * c->S_pad);
    c->conf = color_alloc<unsigned long long>(c, (size_t)c->S_pad);
    c->nonfinite = color_alloc<unsigned long long>(c, 1);
    c->part = color_alloc<float2>(c, (size_t)2 * n * K * kMaxChunks);
    c->shift = color_alloc<float>(c, (size_t)2 * n * K);
    c->rsum = color_alloc<float>(c, (size_t)n * c->S_pad);
    c->t_dev = color_alloc<int32_t>(c, 1);
    c->timeouts = color_alloc<unsigned long long>(c, 1);
    c->sched = color_alloc<float4>(c, (size_t)prm->steps);
    // columns per lane of the gather: as many as keep four blocks per SM, else
    // as many as fit the slab; graphs above 1600 nodes gather directly
    const int64_t Ccols = (int64_t)K * c->S_pad;
    const int64_t row_bytes = 128;   // one float per lane
    for (int vec : {4, 2, 1}) {
        if (Ccols % (32 * vec) != 0) continue;
        if ((int64_t)n * row_bytes * vec <= 56 * 1024) {
            c->gather_vec = vec;
            break;
        }
    }
    if (!c->gather_vec) {
        for (int vec : {2, 1}) {
            if (Ccols % (32 * vec) == 0 && (int64_t)n * row_bytes * vec <= kGatherSlabMax) {
                c->gather_vec = vec;
                break;
            }
        }
    }
    {
        const double density = (double)c->nnz / ((double)n * (double)n);
        if (n >= kTcMinNodes && n <= kTcMaxNodes && density >= kTcMinDensity && Ccols % 64 == 0)
            c->tc_nt = Ccols % 128 == 0 ? 128 : 64;
    }
    if (c->tc_nt) {
        c->gather_vec = 0;
        c->n_pad = (n + 127) / 128 * 128;
        c->A16 = color_alloc<__half>(c, (size_t)c->n_pad * c->n_pad);
        c->hi = color_alloc<__half>(c, (size_t)Ccols * c->n_pad);
        c->lo = color_alloc<__half>(c, (size_t)Ccols * c->n_pad);
        c->tmaps = color_alloc<unsigned char>(c, 3 * sizeof(CUtensorMap));
        c->Y = color_alloc<float>(c, nks);
        if (!c->A16 || !c->hi || !c->lo || !c->tmaps || !c->Y) {
            color_free(c);
            return cfail(QQA_ENOMEM, "device allocation for the tensor-core neighbour sums failed");
        }
        alignas(64) CUtensorMap maps[3];
        const uint64_t rb = (uint64_t)c->n_pad * 2;
        int er = encode_tmap_f16_2d(&maps[0], c->A16, (uint64_t)c->n_pad, (uint64_t)c->n_pad, rb, 64, 128);
        if (!er) er = encode_tmap_f16_2d(&maps[1], c->hi, (uint64_t)c->n_pad, (uint64_t)Ccols, rb, 64, (uint32_t)c->tc_nt);
        if (!er) er = encode_tmap_f16_2d(&maps[2], c->lo, (uint64_t)c->n_pad, (uint64_t)Ccols, rb, 64, (uint32_t)c->tc_nt);
        if (er) {
            color_free(c);
            return cfail(QQA_ECUDA, "tensor map encoding failed (%d)", er);
        }
        std::vector<uint16_t> a16((size_t)c->n_pad * c->n_pad, 0);
        for (int32_t i = 0; i < n; ++i)
            for (int32_t e = row_ptr[i]; e < row_ptr[i + 1]; ++e) a16[(size_t)i * c->n_pad + col[e]] = 0x3C00u;   // fp16 1.0
        cudaError_t ea = cudaMemcpy(c->A16, a16.data(), a16.size() * sizeof(uint16_t), cudaMemcpyHostToDevice);
        if (ea == cudaSuccess) ea = cudaMemcpy(c->tmaps, maps, sizeof maps, cudaMemcpyHostToDevice);
        if (ea == cudaSuccess) ea = cudaMemset(c->hi, 0, (size_t)Ccols * c->n_pad * sizeof(__half));
        if (ea == cudaSuccess) ea = cudaMemset(c->lo, 0, (size_t)Ccols * c->n_pad * sizeof(__half));
        if (ea == cudaSuccess)
            ea = cudaFuncSetAttribute(color_gather_tc_kernel<128>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                      tc_smem_bytes(128));
        if (ea == cudaSuccess)
            ea = cudaFuncSetAttribute(color_gather_tc_kernel<64>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                      tc_smem_bytes(64));
        if (ea != cudaSuccess) {
            (void)cudaGetLastError();
            color_free(c);
            return cfail(QQA_ECUDA, "tensor-core neighbour sums setup: %s", cudaGetErrorString(ea));
        }
    }
    if (c->gather_vec) {
        c->Y = color_alloc<float>(c, nks);
        cudaError_t ea = cudaFuncSetAttribute(color_gather_kernel<4>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                              kGatherSlabMax);
        if (ea == cudaSuccess)
            ea = cudaFuncSetAttribute(color_gather_kernel<2>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                      kGatherSlabMax);
        if (ea == cudaSuccess)
            ea = cudaFuncSetAttribute(color_gather_kernel<1>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                      kGatherSlabMax);
        if (ea != cudaSuccess) {
            (void)cudaGetLastError();
            color_free(c);
            return cfail(QQA_ECUDA, "cannot raise the shared-memory limit of the gather kernel");
        }
    }
    if (!c->part || !c->shift || !c->rsum || !c->t_dev || !c->timeouts || !c->sched || (c->gather_vec && !c->Y) || !c->rp || !c->col || !c->W || !c->m || !c->v || !c->sig[0] || !c->sig[1] ||
        !c->x || !c->conf ||
        !c->nonfinite) {
        color_free(c);
        return cfail(QQA_ENOMEM, "device allocation for the colouring state failed");
    }
    cudaError_t e = cudaMemcpyAsync(c->rp, row_ptr, sizeof(int32_t) * ((size_t)n + 1), cudaMemcpyHostToDevice, c->st);
    if (e == cudaSuccess && c->nnz > 0)
        e = cudaMemcpyAsync(c->col, col, sizeof(int32_t) * (size_t)c->nnz, cudaMemcpyHostToDevice, c->st);
    if (e == cudaSuccess) e = cudaMemsetAsync(c->m, 0, nks * sizeof(float), c->st);
    if (e == cudaSuccess) e = cudaMemsetAsync(c->v, 0, nks * sizeof(float), c->st);
    if (e == cudaSuccess) e = cudaMemsetAsync(c->sig[0], 0, nks * sizeof(float), c->st);
    if (e == cudaSuccess) e = cudaMemsetAsync(c->sig[1], 0, nks * sizeof(float), c->st);
    if (e == cudaSuccess) e = cudaMemsetAsync(c->nonfinite, 0, sizeof(unsigned long long), c->st);
    if (e == cudaSuccess) e = cudaMemsetAsync(c->rsum, 0, sizeof(float) * (size_t)n * c->S_pad, c->st);
    if (e == cudaSuccess) e = cudaMemsetAsync(c->part, 0, sizeof(float2) * (size_t)2 * n * K * kMaxChunks, c->st);
    if (e == cudaSuccess) e = cudaMemsetAsync(c->shift, 0, sizeof(float) * (size_t)2 * n * K, c->st);
    if (e == cudaSuccess) e = cudaMemsetAsync(c->t_dev, 0, sizeof(int32_t), c->st);
    if (e == cudaSuccess) e = cudaMemsetAsync(c->timeouts, 0, sizeof(unsigned long long), c->st);
    // per-step scalars: linear gamma schedule (App. C.2), AdamW bias corrections
    std::vector<float4> sched((size_t)prm->steps);
    for (int32_t t = 0; t < prm->steps; ++t) {
        const double gamma = prm->steps > 1 ? (double)prm->gamma_min + ((double)prm->gamma_max - (double)prm->gamma_min) *
                                                                           (double)t / (double)(prm->steps - 1)
                                            : (double)prm->gamma_min;
        const double bc1 = 1.0 - std::pow((double)prm->beta1, (double)(t + 1));
        const double bc2 = 1.0 - std::pow((double)prm->beta2, (double)(t + 1));
        sched[t] = make_float4((float)(gamma * (-c->cK * (double)prm->a_ent * (double)K)),
                               (float)((double)prm->lr / bc1), (float)(1.0 / std::sqrt(bc2)), 0.0f);
    }
    if (e == cudaSuccess)
        e = cudaMemcpyAsync(c->sched, sched.data(), sizeof(float4) * sched.size(), cudaMemcpyHostToDevice, c->st);
    if (e == cudaSuccess) e = cudaStreamSynchronize(c->st);
    if (e != cudaSuccess) {
        color_free(c);
        return cfail(QQA_ECUDA, "colouring state upload: %s", cudaGetErrorString(e));
    }
    const int64_t total = (int64_t)nks;
    color_init_kernel<<<(unsigned)((total + 255) / 256), 256, 0, c->st>>>(
        n, K, c->S, c->S_pad, (uint32_t)(prm->seed & 0xffffffffu), (uint32_t)(prm->seed >> 32), c->W);
    if (cudaGetLastError() != cudaSuccess) {
        color_free(c);
        return cfail(QQA_ECUDA, "colouring init launch failed");
    }
    add_launches(1);
    rc = color_launch_sigma(c, 0);
    if (rc != QQA_OK) {
        color_free(c);
        return rc;
    }
    *out = c;
    return QQA_OK;
}

extern "C" void qqa_color_destroy(qqa_color *c) { color_free(c); }

extern "C" int qqa_color_steps(qqa_color *c, int32_t nsteps, int32_t *done)
{
    if (!c) return cfail(QQA_EINVAL, "colouring handle is NULL");
    if (nsteps < 0) return cfail(QQA_EINVAL, "nsteps must be >= 0");
    const int32_t todo = std::min<int32_t>(nsteps, c->prm.steps - c->t);
    const int rc = color_run(c, todo);
    if (rc != QQA_OK) return rc;
    if (done) *done = todo;
    return QQA_OK;
}

extern "C" int qqa_color_sync(qqa_color *c)
{
    if (!c) return cfail(QQA_EINVAL, "colouring handle is NULL");
    unsigned long long bad = 0, late = 0;
    COLOR_CK(cudaMemcpyAsync(&bad, c->nonfinite, sizeof bad, cudaMemcpyDeviceToHost, c->st));
    COLOR_CK(cudaMemcpyAsync(&late, c->timeouts, sizeof late, cudaMemcpyDeviceToHost, c->st));
    COLOR_CK(cudaStreamSynchronize(c->st));
    if (late) return cfail(QQA_ETIMEOUT, "%llu bounded waits of the tensor-core neighbour sums ran out", late);
    if (bad) return cfail(QQA_ENONFINITE, "%llu non-finite second moments in the colouring state", bad);
    return QQA_OK;
}

extern "C" int qqa_color_debug_set_status(qqa_color *c, uint64_t nonfinite, uint64_t timeouts)
{
    if (!c) return cfail(QQA_EINVAL, "colouring handle is NULL");
    const unsigned long long bad = nonfinite, late = timeouts;
    COLOR_CK(cudaMemcpyAsync(c->nonfinite, &bad, sizeof bad, cudaMemcpyHostToDevice, c->st));
    COLOR_CK(cudaMemcpyAsync(c->timeouts, &late, sizeof late, cudaMemcpyHostToDevice, c->st));
    COLOR_CK(cudaStreamSynchronize(c->st));
    return QQA_OK;
}

extern "C" int qqa_color_step_debug(qqa_color *c, float *grad)
{
    if (!c) return cfail(QQA_EINVAL, "colouring handle is NULL");
    if (!grad) return cfail(QQA_EINVAL, "grad is NULL");
    if (c->t >= c->prm.steps) return cfail(QQA_EINVAL, "the schedule of %d steps is complete", c->prm.steps);
    if (!c->grad) {
        c->grad = color_alloc<float>(c, c->nks());
        if (!c->grad) return cfail(QQA_ENOMEM, "gradient buffer allocation failed");
    }
    const int k = color_enqueue_chunk(c, 1, c->grad, c->st);
    if (k < 0) return k;
    add_launches((unsigned long long)k);
    c->t += 1;
    std::vector<float> buf(c->nks());
    COLOR_CK(cudaMemcpyAsync(buf.data(), c->grad, buf.size() * sizeof(float), cudaMemcpyDeviceToHost, c->st));
    COLOR_CK(cudaStreamSynchronize(c->st));
    for (size_t r = 0; r < (size_t)c->n * c->K; ++r)
        std::memcpy(grad + r * c->S, buf.data() + r * c->S_pad, sizeof(float) * (size_t)c->S);
    return qqa_color_sync(c);
}

extern "C" int qqa_color_get_state(qqa_color *c, float *W, float *m, float *v, int32_t *t)
{
    if (!c) return cfail(QQA_EINVAL, "colouring handle is NULL");
    std::vector<float> buf(c->nks());
    float *dst[3] = {W, m, v};
    const float *src[3] = {c->W, c->m, c->v};
    for (int q = 0; q < 3; ++q) {
        if (!dst[q]) continue;
        COLOR_CK(cudaMemcpyAsync(buf.data(), src[q], buf.size() * sizeof(float), cudaMemcpyDeviceToHost, c->st));
        COLOR_CK(cudaStreamSynchronize(c->st));
        for (size_t r = 0; r < (size_t)c->n * c->K; ++r)
            std::memcpy(dst[q] + r * c->S, buf.data() + r * c->S_pad, sizeof(float) * (size_t)c->S);
    }
    if (t) *t = c->t;
    return QQA_OK;
}

extern "C" int qqa_color_set_state(qqa_color *c, const float *W, const float *m, const float *v, int32_t t)
{
    if (!c) return cfail(QQA_EINVAL, "colouring handle is NULL");
    if (!W || !m || !v) return cfail(QQA_EINVAL, "W, m and v are required");
    if (t < 0 || t > c->prm.steps) return cfail(QQA_EINVAL, "t must be in [0, %d] (got %d)", c->prm.steps, t);
    const size_t count = (size_t)c->n * c->K * c->S;
    for (size_t e = 0; e < count; ++e) {
        if (!(W[e] >= 0.0f && W[e] <= 1.0f)) return cfail(QQA_EINVAL, "W[%zu] = %g is not in [0, 1]", e, (double)W[e]);
        if (!std::isfinite(m[e])) return cfail(QQA_EINVAL, "m[%zu] is not finite", e);
        if (!(v[e] >= 0.0f) || !std::isfinite(v[e])) return cfail(QQA_EINVAL, "v[%zu] = %g is not >= 0", e, (double)v[e]);
    }
    std::vector<float> buf(c->nks(), 0.0f);
    const float *src[3] = {W, m, v};
    float *dst[3] = {c->W, c->m, c->v};
    for (int q = 0; q < 3; ++q) {
        for (size_t r = 0; r < (size_t)c->n * c->K; ++r)
            std::memcpy(buf.data() + r * c->S_pad, src[q] + r * c->S, sizeof(float) * (size_t)c->S);
        COLOR_CK(cudaMemcpyAsync(dst[q], buf.data(), buf.size() * sizeof(float), cudaMemcpyHostToDevice, c->st));
        COLOR_CK(cudaStreamSynchronize(c->st));
    }
    c->t = t;
    COLOR_CK(cudaMemsetAsync(c->nonfinite, 0, sizeof(unsigned long long), c->st));
    color_set_t_kernel<<<1, 1, 0, c->st>>>(c->t_dev, t);
    COLOR_CK(cudaGetLastError());
    add_launches(1);
    return color_launch_sigma(c, t & 1);
}

extern "C" int qqa_color_round(qqa_color *c, int64_t *conflicts, int32_t *best_s, uint8_t *x_all)
{
    if (!c) return cfail(QQA_EINVAL, "colouring handle is NULL");
    if (!conflicts || !best_s) return cfail(QQA_EINVAL, "conflicts and best_s are required");
    const int64_t total = (int64_t)c->n * c->S_pad;
    const unsigned blocks = (unsigned)((total + 255) / 256);
    COLOR_CK(cudaMemsetAsync(c->conf, 0, sizeof(unsigned long long) * (size_t)c->S_pad, c->st));
    color_argmax_kernel<<<blocks, 256, 0, c->st>>>(c->n, c->K, c->S, c->S_pad, c->W, c->x);
    COLOR_CK(cudaGetLastError());
    color_conflict_kernel<<<blocks, 256, 0, c->st>>>(c->n, c->S, c->S_pad, c->rp, c->col, c->x, c->conf);
    COLOR_CK(cudaGetLastError());
    add_launches(2);
    std::vector<unsigned long long> h((size_t)c->S_pad);
    COLOR_CK(cudaMemcpyAsync(h.data(), c->conf, sizeof(unsigned long long) * h.size(), cudaMemcpyDeviceToHost, c->st));
    std::vector<uint8_t> xb;
    if (x_all) {
        xb.resize((size_t)c->n * c->S_pad);
        COLOR_CK(cudaMemcpyAsync(xb.data(), c->x, xb.size(), cudaMemcpyDeviceToHost, c->st));
    }
    const int rc = qqa_color_sync(c);
    if (rc != QQA_OK) return rc;
    int32_t best = 0;
    for (int32_t s = 0; s < c->S; ++s) {
        conflicts[s] = (int64_t)h[s];
        if (h[s] < h[best]) best = s;
    }
    *best_s = best;
    if (x_all)
        for (int32_t i = 0; i < c->n; ++i) std::memcpy(x_all + (size_t)i * c->S, xb.data() + (size_t)i * c->S_pad, c->S);
    return QQA_OK;
}

extern "C" int qqa_color_info(const qqa_color *c, int32_t *n, int32_t *K, int32_t *S, int32_t *t)
{
    if (!c) return cfail(QQA_EINVAL, "colouring handle is NULL");
    if (n) *n = c->n;
    if (K) *K = c->K;
    if (S) *S = c->S;
    if (t) *t = c->t;
    return QQA_OK;
}
