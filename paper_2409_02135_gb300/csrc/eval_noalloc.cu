// eval_noalloc.cu -- projection rounding and exact costs of a replica state
// that lives in the caller's device memory, without any device allocation.
//
// Who needs it: callers that must not allocate device memory when they ask
// for an evaluation. A serving loop that budgets HBM up front cannot let a
// request fail on, or stall behind, an allocation (cudaMalloc can synchronise
// the device); a host framework that owns every device byte through its own
// allocator cannot hand allocation to a library. Such a caller passes device
// pointers for the graph, the state and the outputs, and this entry point
// works in a fixed scratch array that is part of the library image.
//
// The scratch array is a file-scope __device__ object: every GPU that loads
// the library holds it (a little over 4 MiB) until the process exits, and
// every call shares it, so calls whose work overlaps on the GPU race with one
// another. Each call clears the counters it accumulates into before using
// them; the bit array is fully rewritten for the rows a call covers.
//
// Host code cannot use the array's name as a device address (in host code it
// names a host-side stand-in), so the first call on each device asks the
// runtime for the device address with cudaGetSymbolAddress, with that device
// current, and caches it together with the identity of the CUDA context it
// belongs to: after cudaDeviceReset the device gets a new context (and the
// library image a new address), and the next call looks the address up again
// instead of using the stale one. A call that looks the address up should
// come before any stream capture begins.
#include <algorithm>
#include <cstdio>
#include <mutex>
#include <string>

#include <cuda.h>

#include "../../include/qqa.h"

namespace {

constexpr int kNoAllocMaxS = 1024;                 // replicas
constexpr size_t kNoAllocBitWords = size_t(1) << 20;   // n * ceil(S / 32) words of rounded replicas
constexpr int kMaxDevices = 64;

struct NoAllocScratch {
    unsigned long long counts[3 * kNoAllocMaxS];   // per replica: size, inside edges, cut weight
    unsigned int bits[kNoAllocBitWords];           // bit s%32 of word [i][s/32] = x_is
};

__device__ __align__(256) NoAllocScratch g_noalloc_scratch;

std::mutex g_mu;
NoAllocScratch *g_scratch_addr[kMaxDevices] = {};
unsigned long long g_scratch_ctx[kMaxDevices] = {};   // unique id of the context the address is valid in

// Unique id of the calling thread's current CUDA context (driver entry points
// looked up through the runtime, so the library needs no link to libcuda).
bool current_context_id(unsigned long long *id)
{
    using GetCurrent = CUresult (*)(CUcontext *);
    using GetId = CUresult (*)(CUcontext, unsigned long long *);
    static GetCurrent get_current = nullptr;
    static GetId get_id = nullptr;
    static std::once_flag once;
    std::call_once(once, [] {
        cudaDriverEntryPointQueryResult q;
        void *p = nullptr;
        if (cudaGetDriverEntryPointByVersion("cuCtxGetCurrent", &p, 12000, cudaEnableDefault, &q) == cudaSuccess &&
            q == cudaDriverEntryPointSuccess)
            get_current = reinterpret_cast<GetCurrent>(p);
        if (cudaGetDriverEntryPointByVersion("cuCtxGetId", &p, 12000, cudaEnableDefault, &q) == cudaSuccess &&
            q == cudaDriverEntryPointSuccess)
            get_id = reinterpret_cast<GetId>(p);
        (void)cudaGetLastError();
    });
    CUcontext ctx = nullptr;
    if (!get_current || !get_id || get_current(&ctx) != CUDA_SUCCESS || !ctx) return false;
    return get_id(ctx, id) == CUDA_SUCCESS;
}

thread_local std::string g_noalloc_error;

int noalloc_fail(int code, const char *msg)
{
    g_noalloc_error = msg;
    return code;
}

// x_is = [X[i][s] > 1/2] for s < S, packed 32 replicas to a word; the counters
// are cleared by block 0 (the count kernel runs after this one on the stream).
__global__ void na_bits_kernel(NoAllocScratch *sc, int n, int S, long long ld, const float *__restrict__ X)
{
    const int W = (S + 31) / 32;
    if (blockIdx.x == 0)
        for (int k = threadIdx.x; k < 3 * kNoAllocMaxS; k += blockDim.x) sc->counts[k] = 0ULL;
    const int lane = threadIdx.x & 31;
    const long long warp = (blockIdx.x * (long long)blockDim.x + threadIdx.x) >> 5;
    const long long nwarps = ((long long)gridDim.x * blockDim.x) >> 5;
    for (long long p = warp; p < (long long)n * W; p += nwarps) {
        const long long i = p / W;
        const int w = (int)(p % W);
        const int s = 32 * w + lane;
        const bool x = s < S && X[i * ld + s] > 0.5f;
        const unsigned word = __ballot_sync(0xffffffffu, x);
        if (lane == 0) sc->bits[i * W + w] = word;
    }
}

// Per replica: size = sum_i x_i, inside = #edges i<j with x_i x_j,
// cut = sum_{i<j} w_ij [x_i != x_j]. A block covers `rows` consecutive rows;
// its threads split (row, replica) items and combine in shared memory first.
// The graph comes as device pointers the host cannot inspect: row offsets are
// clamped to [0, nnz] and neighbour indices outside [0, n) are skipped, so a
// malformed graph gives wrong counts but never an out-of-bounds access.
__global__ void na_count_kernel(NoAllocScratch *sc, int n, long long nnz, int S, int rows,
                                const int *__restrict__ row_ptr, const int *__restrict__ col,
                                const int *__restrict__ wt)
{
    __shared__ long long part[3 * kNoAllocMaxS];
    const int W = (S + 31) / 32;
    const int S32 = W * 32;
    for (int k = threadIdx.x; k < 3 * S32; k += blockDim.x) part[k] = 0;
    __syncthreads();
    const int r0 = blockIdx.x * rows;
    const int r1 = min(r0 + rows, n);
    const int splits = max(1, (int)blockDim.x / S32);
    for (int base = threadIdx.x; base < splits * S32; base += blockDim.x) {
        const int s = base % S32;
        const int split = base / S32;
        if (s >= S) continue;
        const int w = s >> 5, b = s & 31;
        long long size = 0, inside = 0, cut = 0;
        for (int i = r0 + split; i < r1; i += splits) {
            const unsigned xi = (sc->bits[(size_t)i * W + w] >> b) & 1u;
            size += xi;
            const long long k0 = max(0LL, min((long long)row_ptr[i], nnz));
            const long long k1 = max(k0, min((long long)row_ptr[i + 1], nnz));
            for (long long k = k0; k < k1; ++k) {
                const int j = col[k];
                if (j <= i || j >= n) continue;
                const unsigned xj = (sc->bits[(size_t)j * W + w] >> b) & 1u;
                inside += (long long)(xi & xj);
                if (xi != xj) cut += wt ? (long long)wt[k] : 1LL;
            }
        }
        if (size) atomicAdd((unsigned long long *)&part[s], (unsigned long long)size);
        if (inside) atomicAdd((unsigned long long *)&part[S32 + s], (unsigned long long)inside);
        if (cut) atomicAdd((unsigned long long *)&part[2 * S32 + s], (unsigned long long)cut);
    }
    __syncthreads();
    for (int s = threadIdx.x; s < S; s += blockDim.x) {
        if (part[s]) atomicAdd(&sc->counts[s], (unsigned long long)part[s]);
        if (part[S32 + s]) atomicAdd(&sc->counts[kNoAllocMaxS + s], (unsigned long long)part[S32 + s]);
        if (part[2 * S32 + s]) atomicAdd(&sc->counts[2 * kNoAllocMaxS + s], (unsigned long long)part[2 * S32 + s]);
    }
}

// One warp: objective, violation, feasibility and energy of every replica and
// the best feasible replica (largest objective, ties -> lowest index).
__global__ void na_finalize_kernel(const NoAllocScratch *sc, int kind, int S, float lambda, long long *obj_out,
                                   long long *viol_out, unsigned char *feas_out, double *energy_out, int *best_out)
{
    const int lane = threadIdx.x;
    long long best_obj = 0;
    int best_s = -1;
    for (int s = lane; s < S; s += 32) {
        const long long size = (long long)sc->counts[s];
        const long long inside = (long long)sc->counts[kNoAllocMaxS + s];
        const long long cut = (long long)sc->counts[2 * kNoAllocMaxS + s];
        long long o, v;
        double e;
        if (kind == QQA_MIS) {
            o = size; v = inside;
            e = -(double)size + (double)lambda * (double)inside;
        } else if (kind == QQA_MAXCLIQUE) {
            o = size; v = size * (size - 1) / 2 - inside;
            e = -(double)size + (double)lambda * (double)v;
        } else {
            o = cut; v = 0;
            e = -(double)cut;
        }
        obj_out[s] = o;
        viol_out[s] = v;
        feas_out[s] = v == 0 ? 1 : 0;
        energy_out[s] = e;
        if (v == 0 && (best_s < 0 || o > best_obj)) { best_obj = o; best_s = s; }
    }
    for (int off = 16; off > 0; off >>= 1) {
        const long long o2 = __shfl_xor_sync(0xffffffffu, best_obj, off);
        const int s2 = __shfl_xor_sync(0xffffffffu, best_s, off);
        if (s2 >= 0 && (best_s < 0 || o2 > best_obj || (o2 == best_obj && s2 < best_s))) { best_obj = o2; best_s = s2; }
    }
    if (lane == 0) *best_out = best_s;
}

}  // namespace

extern "C" const char *qqa_noalloc_last_error(void) { return g_noalloc_error.c_str(); }

extern "C" int qqa_round_eval_noalloc(int32_t kind, int32_t n, int64_t nnz, const int32_t *row_ptr,
                                      const int32_t *col, const int32_t *w, int32_t S, int64_t ld, const float *X,
                                      float lambda,
                                      int64_t *obj, int64_t *viol, uint8_t *feasible, double *energy,
                                      int32_t *best_s, void *stream)
{
    if (kind < QQA_MIS || kind > QQA_MAXCLIQUE) return noalloc_fail(QQA_EINVAL, "unknown problem kind");
    if (n < 1) return noalloc_fail(QQA_EINVAL, "n must be >= 1");
    if (nnz < 0 || nnz >= (int64_t(1) << 31)) return noalloc_fail(QQA_EINVAL, "nnz must be in [0, 2^31)");
    if (S < 1 || S > kNoAllocMaxS) return noalloc_fail(QQA_EINVAL, "S must be in [1, 1024] for the static scratch");
    if (ld < S) return noalloc_fail(QQA_EINVAL, "row stride ld must be >= S");
    if ((size_t)n * (size_t)((S + 31) / 32) > kNoAllocBitWords)
        return noalloc_fail(QQA_EINVAL,
                            "n * ceil(S/32) exceeds the static scratch of 1048576 words (4 MiB); "
                            "use qqa_round_eval, which allocates");
    if (!row_ptr || !col || !X || !obj || !viol || !feasible || !energy || !best_s)
        return noalloc_fail(QQA_EINVAL, "a required pointer is NULL (only w may be NULL)");
    if (w && kind != QQA_MAXCUT) return noalloc_fail(QQA_EINVAL, "edge weights are only defined for max-cut");

    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= kMaxDevices) {
        (void)cudaGetLastError();
        return noalloc_fail(QQA_ECUDA, "no usable current CUDA device");
    }
    NoAllocScratch *sc = nullptr;
    {
        std::lock_guard<std::mutex> lock(g_mu);
        unsigned long long ctx_id = 0;
        if (!g_scratch_addr[dev] || !current_context_id(&ctx_id) || ctx_id != g_scratch_ctx[dev]) {
            // first call on this device, or its context changed (or cannot be
            // identified): the runtime creates the context if needed, then the
            // address is looked up for it
            void *p = nullptr;
            const cudaError_t e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
            if (e != cudaSuccess || !p) {
                (void)cudaGetLastError();
                return noalloc_fail(QQA_ECUDA, "cudaGetSymbolAddress of the static scratch failed");
            }
            g_scratch_addr[dev] = static_cast<NoAllocScratch *>(p);
            g_scratch_ctx[dev] = current_context_id(&ctx_id) ? ctx_id : 0;
        }
        sc = g_scratch_addr[dev];
    }
    cudaStream_t st = (cudaStream_t)stream;
    const long long pairs = (long long)n * ((S + 31) / 32);
    const int bits_grid = (int)std::min<long long>((pairs * 32 + 255) / 256, 4096);
    na_bits_kernel<<<bits_grid, 256, 0, st>>>(sc, n, S, (long long)ld, X);
    const int rows = 16;
    na_count_kernel<<<(n + rows - 1) / rows, 256, 0, st>>>(sc, n, (long long)nnz, S, rows, row_ptr, col, w);
    na_finalize_kernel<<<1, 32, 0, st>>>(sc, kind, S, lambda, reinterpret_cast<long long *>(obj),
                                         reinterpret_cast<long long *>(viol), feasible, energy, best_s);
    const cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return noalloc_fail(QQA_ECUDA, cudaGetErrorString(e));
    return QQA_OK;
}
