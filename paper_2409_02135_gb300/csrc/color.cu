// color.cu -- categorical PQQA for graph colouring (App. B, App. C.4, App. D.1).
//
// State of one instance: W[i][k][s] in [0,1] for node i < n, colour k < K and
// replica s < S, with the AdamW moments m, v in the same layout, and the
// categorical relaxation sigma = W / sum_k W (Clamp-normalise, App. C.4; the
// clamp is the identity because every update ends with the projection to
// [0,1]). Rows of one (i, k) are S_pad = S rounded up to 32 floats long, so a
// warp reads 128 contiguous bytes of one colour plane.
//
// One step (color_step_kernel, one block per node, replicas across threads):
//   statistics  mean_ik, STD_ik = sqrt(var_ik + eps) of sigma over replicas (Eq. 10)
//   gradient    g_ik = sum_{j in N(i)} sigma_jk                       relaxed conflicts
//                    + gamma_t (-c_K a K) (K sigma_ik - 1)^(a-1)      entropy s_K (App. B)
//                    - alpha (sigma_ik - mean_ik) / STD_ik            communication (Eq. 10)
//               dR/dW_ik = (g_ik - sum_k' sigma_ik' g_ik') / sum_k W_ik   (Clamp-normalise chain rule)
//   update      AdamW with decoupled decay, + sqrt(2 lr T) xi, projection to [0,1]
//   relaxation  sigma' = W' / sum_k W' (a zero row: 1/K), into the other buffer
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
#include <vector>

#include "../../include/qqa.h"
#include "qqa_internal.cuh"

namespace qqa {
int set_error(int code, const char *msg);
int check_unit_graph(int32_t n, const int32_t *rp, const int32_t *col);
void add_launches(unsigned long long k);
}  // namespace qqa

using namespace qqa;

namespace {

constexpr int kColorThreads = 256;       // block of the step kernel (replicas strided over it)
constexpr int kColorWarps = kColorThreads / 32;

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

// Per-step scalars, computed on the host in double and rounded once.
struct ColorStepArgs {
    int32_t n, K, S, S_pad, t, half_pow;
    float ent_coef;       // gamma_t * (-c_K a K)
    float step_size;      // lr / (1 - b1^(t+1))
    float inv_sqrt_bc2;   // 1 / sqrt(1 - b2^(t+1))
    float decay;          // 1 - lr * weight_decay
    float b1, b2, adam_eps, alpha, comm_eps, noise_scale;
    uint32_t seed_lo, seed_hi;
};

// Sum of v[k] over the block for every k < KMAX; every thread gets the totals in out[].
template <int KMAX>
__device__ __forceinline__ void block_sum(float (&v)[KMAX], float (*part)[KMAX], float *out, int K)
{
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
#pragma unroll
    for (int k = 0; k < KMAX; ++k) {
        if (k >= K) break;
        float x = v[k];
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) x += __shfl_xor_sync(0xffffffffu, x, o);
        if (lane == 0) part[warp][k] = x;
    }
    __syncthreads();
    if (threadIdx.x < K) {
        float acc = 0.0f;
        for (int w = 0; w < (int)(blockDim.x >> 5); ++w) acc += part[w][threadIdx.x];
        out[threadIdx.x] = acc;
    }
    __syncthreads();
}

// Standard normal of (counter row, replica s, step t): element s mod 4 of the
// Box-Muller quad of Philox block (row, s/4, t, 1), the binary method's stream.
__device__ __forceinline__ float color_gauss(uint32_t lo, uint32_t hi, uint32_t row, int s, uint32_t t)
{
    const U4 r = philox10(U4{row, (uint32_t)(s >> 2), t, 1u}, lo, hi);
    const int e = s & 3;
    float z0, z1;
    if (e < 2) box_muller(r.x, r.y, z0, z1);
    else box_muller(r.z, r.w, z0, z1);
    return (e & 1) ? z1 : z0;
}

template <int KMAX>
__global__ void __launch_bounds__(kColorThreads)
color_step_kernel(ColorStepArgs a, const int32_t *__restrict__ rp, const int32_t *__restrict__ col,
                  const float *__restrict__ sig_cur, float *__restrict__ sig_next, float *__restrict__ W,
                  float *__restrict__ M, float *__restrict__ V, float *__restrict__ grad_dbg,
                  unsigned long long *__restrict__ nonfinite)
{
    __shared__ float part[kColorWarps][KMAX];
    __shared__ float sh_mean[KMAX], sh_ss[KMAX];
    const int K = a.K, S = a.S;
    const size_t plane = (size_t)a.S_pad, node = (size_t)K * plane;
    const float inv_S = 1.0f / (float)S;
    const float om_b1 = 1.0f - a.b1, om_b2 = 1.0f - a.b2;
    const float fK = (float)K;

    for (int i = blockIdx.x; i < a.n; i += gridDim.x) {
        const float *__restrict__ sig_i = sig_cur + (size_t)i * node;
        // population mean and variance of sigma_ik over the replicas (two passes)
        float acc[KMAX];
#pragma unroll
        for (int k = 0; k < KMAX; ++k) acc[k] = 0.0f;
        for (int s = threadIdx.x; s < S; s += blockDim.x) {
#pragma unroll
            for (int k = 0; k < KMAX; ++k)
                if (k < K) acc[k] += sig_i[k * plane + s];
        }
        block_sum<KMAX>(acc, part, sh_mean, K);
        float mean[KMAX];
#pragma unroll
        for (int k = 0; k < KMAX; ++k) {
            mean[k] = k < K ? sh_mean[k] * inv_S : 0.0f;
            acc[k] = 0.0f;
        }
        for (int s = threadIdx.x; s < S; s += blockDim.x) {
#pragma unroll
            for (int k = 0; k < KMAX; ++k)
                if (k < K) {
                    const float d = sig_i[k * plane + s] - mean[k];
                    acc[k] = fmaf(d, d, acc[k]);
                }
        }
        block_sum<KMAX>(acc, part, sh_ss, K);
        float comm[KMAX];   // -alpha / STD_ik
#pragma unroll
        for (int k = 0; k < KMAX; ++k)
            comm[k] = k < K ? -a.alpha / sqrtf(fmaf(sh_ss[k], inv_S, a.comm_eps)) : 0.0f;

        const int e0 = rp[i], e1 = rp[i + 1];
        for (int s = threadIdx.x; s < S; s += blockDim.x) {
            float sg[KMAX], y[KMAX];
            float wsum = 0.0f;
#pragma unroll
            for (int k = 0; k < KMAX; ++k) {
                sg[k] = k < K ? sig_i[k * plane + s] : 0.0f;
                wsum += k < K ? W[(size_t)i * node + k * plane + s] : 0.0f;
                y[k] = 0.0f;
            }
            // relaxed conflicts: sum of the neighbours' sigma of the same colour
            for (int e = e0; e < e1; ++e) {
                const float *__restrict__ sj = sig_cur + (size_t)__ldg(col + e) * node + s;
#pragma unroll
                for (int k = 0; k < KMAX; ++k)
                    if (k < K) y[k] += sj[k * plane];
            }
            // dR/dsigma, then the chain rule through W / sum W
            float dot = 0.0f;
#pragma unroll
            for (int k = 0; k < KMAX; ++k) {
                if (k >= K) break;
                const float u = fmaf(fK, sg[k], -1.0f);
                const float u2 = u * u;
                float upow = u;
                for (int h = 0; h < a.half_pow; ++h) upow *= u2;
                float g = fmaf(a.ent_coef, upow, y[k]);
                g = fmaf(comm[k], sg[k] - mean[k], g);
                y[k] = g;
                dot = fmaf(sg[k], g, dot);
            }
            const float inv_w = wsum > 0.0f ? 1.0f / wsum : 0.0f;
            float wn[KMAX];
            float nsum = 0.0f, vsum = 0.0f;
#pragma unroll
            for (int k = 0; k < KMAX; ++k) {
                if (k >= K) break;
                const size_t idx = (size_t)i * node + k * plane + s;
                const float g = (y[k] - dot) * inv_w;
                if (grad_dbg) grad_dbg[idx] = g;
                const float mn = fmaf(a.b1, M[idx], om_b1 * g);
                const float vn = fmaf(a.b2, V[idx], om_b2 * (g * g));
                const float denom = fmaf(sqrtf(vn), a.inv_sqrt_bc2, a.adam_eps);
                float q = W[idx] * a.decay;
                q = fmaf(-a.step_size, mn / denom, q);
                const float xi = a.noise_scale != 0.0f
                                     ? color_gauss(a.seed_lo, a.seed_hi, (uint32_t)(i * K + k), s, (uint32_t)a.t)
                                     : 0.0f;
                const float w = __saturatef(fmaf(a.noise_scale, xi, q));
                M[idx] = mn;
                V[idx] = vn;
                W[idx] = w;
                wn[k] = w;
                nsum += w;
                vsum += vn;
            }
            if (!(vsum <= 3.0e38f)) atomicAdd(nonfinite, 1ULL);
            const float inv_n = nsum > 0.0f ? 1.0f / nsum : 0.0f;
            float *__restrict__ out = sig_next + (size_t)i * node + s;
#pragma unroll
            for (int k = 0; k < KMAX; ++k) {
                if (k >= K) break;
                out[k * plane] = nsum > 0.0f ? wn[k] * inv_n : 1.0f / fK;
            }
        }
        __syncthreads();   // shared statistics are rewritten by the next node
    }
}

// sigma = W / sum_k W for every (i, s) (1/K for a zero row).
__global__ void color_sigma_kernel(int32_t n, int32_t K, int32_t S, int32_t S_pad, const float *__restrict__ W,
                                   float *__restrict__ sig)
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

using ColorFn = void (*)(ColorStepArgs, const int32_t *, const int32_t *, const float *, float *, float *, float *,
                         float *, float *, unsigned long long *);

ColorFn color_kernel_for(int K)
{
    if (K <= 4) return color_step_kernel<4>;
    if (K <= 8) return color_step_kernel<8>;
    if (K <= 16) return color_step_kernel<16>;
    return color_step_kernel<32>;
}

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
    uint8_t *x = nullptr;
    unsigned long long *conf = nullptr, *nonfinite = nullptr;
    std::vector<void *> owned;

    size_t nks() const { return (size_t)n * (size_t)K * (size_t)S_pad; }
};

static void color_free(qqa_color *c)
{
    if (!c) return;
    if (c->st) cudaStreamSynchronize(c->st);
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

static int color_launch_sigma(qqa_color *c, int which)
{
    const int64_t total = (int64_t)c->n * c->S_pad;
    color_sigma_kernel<<<(unsigned)((total + 255) / 256), 256, 0, c->st>>>(c->n, c->K, c->S, c->S_pad, c->W,
                                                                        c->sig[which]);
    COLOR_CK(cudaGetLastError());
    add_launches(1);
    return QQA_OK;
}

static int color_launch_step(qqa_color *c, float *grad_dbg)
{
    const qqa_params &p = c->prm;
    const int t = c->t;
    ColorStepArgs a{};
    a.n = c->n;
    a.K = c->K;
    a.S = c->S;
    a.S_pad = c->S_pad;
    a.t = t;
    a.half_pow = (p.a_ent - 2) / 2;
    const double gamma = p.steps > 1 ? (double)p.gamma_min + ((double)p.gamma_max - (double)p.gamma_min) * (double)t /
                                                                 (double)(p.steps - 1)
                                     : (double)p.gamma_min;
    a.ent_coef = (float)(gamma * (-c->cK * (double)p.a_ent * (double)c->K));
    const double bc1 = 1.0 - std::pow((double)p.beta1, (double)(t + 1));
    const double bc2 = 1.0 - std::pow((double)p.beta2, (double)(t + 1));
    a.step_size = (float)((double)p.lr / bc1);
    a.inv_sqrt_bc2 = (float)(1.0 / std::sqrt(bc2));
    a.decay = (float)(1.0 - (double)p.lr * (double)p.weight_decay);
    a.b1 = p.beta1;
    a.b2 = p.beta2;
    a.adam_eps = p.adam_eps;
    a.alpha = p.alpha_comm;
    a.comm_eps = p.comm_eps;
    a.noise_scale = (float)std::sqrt(2.0 * (double)p.lr * (double)p.temperature);
    a.seed_lo = (uint32_t)(p.seed & 0xffffffffu);
    a.seed_hi = (uint32_t)(p.seed >> 32);
    const int cur = t & 1;
    const unsigned grid = (unsigned)std::min<int64_t>(c->n, (int64_t)c->sms * 16);
    const int threads = std::min(kColorThreads, c->S_pad);
    color_kernel_for(c->K)<<<grid, threads, 0, c->st>>>(a, c->rp, c->col, c->sig[cur], c->sig[cur ^ 1], c->W, c->m,
                                                      c->v, grad_dbg, c->nonfinite);
    COLOR_CK(cudaGetLastError());
    add_launches(1);
    c->t = t + 1;
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
    if (!c->rp || !c->col || !c->W || !c->m || !c->v || !c->sig[0] || !c->sig[1] || !c->x || !c->conf ||
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
    for (int32_t k = 0; k < todo; ++k) {
        const int rc = color_launch_step(c, nullptr);
        if (rc != QQA_OK) return rc;
    }
    if (done) *done = todo;
    return QQA_OK;
}

extern "C" int qqa_color_sync(qqa_color *c)
{
    if (!c) return cfail(QQA_EINVAL, "colouring handle is NULL");
    unsigned long long bad = 0;
    COLOR_CK(cudaMemcpyAsync(&bad, c->nonfinite, sizeof bad, cudaMemcpyDeviceToHost, c->st));
    COLOR_CK(cudaStreamSynchronize(c->st));
    if (bad) return cfail(QQA_ENONFINITE, "%llu non-finite second moments in the colouring state", bad);
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
    int rc = color_launch_step(c, c->grad);
    if (rc != QQA_OK) return rc;
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
