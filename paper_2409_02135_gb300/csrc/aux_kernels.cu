// aux_kernels.cu -- everything around the fused step: initial state, the
// clique column sums, step-counter advance, projection rounding with exact
// integer costs, and state import/export for checkpoints and tests.
#include <algorithm>

#include "qqa_internal.cuh"

namespace qqa {

// ---------------------------------------------------------------------------
// Initial state (the paper leaves it open): p ~ U(0,1] from Philox keyed by
// (seed, node, replica quad, step 0, tag 0); m = v = 0.
// ---------------------------------------------------------------------------
template <typename T>
__global__ void init_kernel(const InstDesc *__restrict__ descs, int32_t slot)
{
    const InstDesc &d = descs[slot];
    if (d.S_pad == 1) {   // one replica per node: element 0 of each node's first quad
        for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < d.n; i += gridDim.x * blockDim.x) {
            float u[4];
            unif4(d.seed_lo, d.seed_hi, (uint32_t)i, 0u, u);
            if (sizeof(T) == 4) {
                reinterpret_cast<float *>(d.X[0])[i] = u[0];
                reinterpret_cast<float *>(d.m)[i] = 0.0f;
                reinterpret_cast<float *>(d.v)[i] = 0.0f;
            } else {
                d.master[i] = u[0];
                reinterpret_cast<__nv_bfloat16 *>(d.X[0])[i] = __float2bfloat16_rn(u[0]);
                reinterpret_cast<__nv_bfloat16 *>(d.m)[i] = __float2bfloat16_rn(0.0f);
                reinterpret_cast<__nv_bfloat16 *>(d.v)[i] = __float2bfloat16_rn(0.0f);
            }
        }
        return;
    }
    const int quads = d.S_pad / 4;
    const long long total = (long long)d.n * quads;
    for (long long idx = blockIdx.x * (long long)blockDim.x + threadIdx.x; idx < total;
         idx += (long long)gridDim.x * blockDim.x) {
        const int i = (int)(idx / quads);
        const int q = (int)(idx % quads);
        float u[4];
        unif4(d.seed_lo, d.seed_hi, (uint32_t)i, (uint32_t)q, u);
        const size_t e = (size_t)i * d.S_pad + 4 * q;
        if (sizeof(T) == 4) {
            *reinterpret_cast<float4 *>(reinterpret_cast<float *>(d.X[0]) + e) = make_float4(u[0], u[1], u[2], u[3]);
            *reinterpret_cast<float4 *>(reinterpret_cast<float *>(d.m) + e) = make_float4(0.f, 0.f, 0.f, 0.f);
            *reinterpret_cast<float4 *>(reinterpret_cast<float *>(d.v) + e) = make_float4(0.f, 0.f, 0.f, 0.f);
        } else {
            *reinterpret_cast<float4 *>(d.master + e) = make_float4(u[0], u[1], u[2], u[3]);
            __nv_bfloat16 *xb = reinterpret_cast<__nv_bfloat16 *>(d.X[0]) + e;
            const __nv_bfloat162 a = __floats2bfloat162_rn(u[0], u[1]);
            const __nv_bfloat162 b = __floats2bfloat162_rn(u[2], u[3]);
            reinterpret_cast<__nv_bfloat162 *>(xb)[0] = a;
            reinterpret_cast<__nv_bfloat162 *>(xb)[1] = b;
            const __nv_bfloat162 z = __floats2bfloat162_rn(0.f, 0.f);
            reinterpret_cast<__nv_bfloat162 *>(reinterpret_cast<__nv_bfloat16 *>(d.m) + e)[0] = z;
            reinterpret_cast<__nv_bfloat162 *>(reinterpret_cast<__nv_bfloat16 *>(d.m) + e)[1] = z;
            reinterpret_cast<__nv_bfloat162 *>(reinterpret_cast<__nv_bfloat16 *>(d.v) + e)[0] = z;
            reinterpret_cast<__nv_bfloat162 *>(reinterpret_cast<__nv_bfloat16 *>(d.v) + e)[1] = z;
        }
    }
}

void launch_init(const InstDesc *descs, int32_t slot, int32_t n, int32_t S_pad, int32_t prec, cudaStream_t st)
{
    const long long total = (long long)n * (S_pad == 1 ? 1 : S_pad / 4);
    const int block = 256;
    const int grid = (int)((total + block - 1) / block < 65535 ? (total + block - 1) / block : 65535);
    if (prec == kFP32) init_kernel<float><<<grid, block, 0, st>>>(descs, slot);
    else init_kernel<__nv_bfloat16><<<grid, block, 0, st>>>(descs, slot);
}

// ---------------------------------------------------------------------------
// Max-clique column sums cs_s = sum_i p_is (the Sum_i p_i term of Eq. 24) of
// one state, always in the same order, so that clique trajectories do not
// depend on how rows were scheduled: a 1024-thread block covers 32
// consecutive replicas (one per lane); warp w sums rows w, w + 32, w + 64, ...
// in order, then lane s of warp 0 adds the 32 warp sums in warp order.
// blockIdx.y indexes the slot list (or the single slot slot0).
// after = 1: the state p^{t+1} written by step t = d.t + r (skipped once the
// instance has finished); after = 0: the current state p^{d.t}.
// ---------------------------------------------------------------------------
__global__ void __launch_bounds__(1024) colsum_kernel(const InstDesc *__restrict__ descs,
                                                      const int32_t *__restrict__ slots, int32_t slot0, int32_t r,
                                                      int32_t after, int32_t prec)
{
    __shared__ float part[32][33];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const InstDesc &d = descs[slots ? slots[blockIdx.y] : slot0];
    const int t = d.t + r;
    if (after && t >= d.K) return;                  // block-uniform
    if ((int)blockIdx.x * 32 >= d.S_pad) return;    // block-uniform
    const int ts = after ? t + 1 : d.t;
    const float *src = prec == kFP32 ? reinterpret_cast<const float *>(d.X[ts & 1]) : d.master;
    const int s = blockIdx.x * 32 + lane;
    float acc = 0.0f;
    if (s < d.S_pad)
        for (int i = warp; i < d.n; i += 32) acc += src[(size_t)i * d.S_pad + s];
    part[warp][lane] = acc;
    __syncthreads();
    if (warp == 0 && s < d.S_pad) {
        float tot = 0.0f;
        for (int w = 0; w < 32; ++w) tot += part[w][lane];
        d.colsum[s] = tot;
    }
}

void launch_colsum(const InstDesc *descs, const int32_t *slots, int32_t count, int32_t slot0, int32_t S_max_pad,
                   int32_t prec, int32_t r, int32_t after, cudaStream_t st)
{
    const dim3 grid((unsigned)((S_max_pad + 31) / 32), (unsigned)(slots ? count : 1));
    colsum_kernel<<<grid, 1024, 0, st>>>(descs, slots, slot0, r, after, prec);
}

// Step counters move forward once per chunk: t = min(t + nsteps, K).
__global__ void advance_kernel(InstDesc *__restrict__ descs, int32_t capacity, int32_t nsteps)
{
    const int k = blockIdx.x * blockDim.x + threadIdx.x;
    if (k >= capacity) return;
    InstDesc &d = descs[k];
    if (!d.active) return;
    const int t = d.t + nsteps;
    d.t = t < d.K ? t : d.K;
}

void launch_advance(InstDesc *descs, int32_t capacity, int32_t nsteps, cudaStream_t st)
{
    advance_kernel<<<(capacity + 127) / 128, 128, 0, st>>>(descs, capacity, nsteps);
}

// Per-step scalars of the next `nsteps` steps of every active slot, computed
// once here instead of in every thread of the step kernel:
//   gamma_t = gamma_min + (gamma_max - gamma_min) t / (K - 1)   (linear schedule, App. C.2)
//   x = gamma_t * (-2a)   (coefficient of (2p - 1)^(a-1) in the gradient, Eq. 7)
//   y = lr / (1 - b1^(t+1)),  z = 1 / sqrt(1 - b2^(t+1))   (AdamW bias corrections;
//   1 - b^k = -expm1(k log1p(b - 1)) avoids cancellation, b - 1 is exact for b in [0.5, 1))
__global__ void prepare_kernel(const InstDesc *__restrict__ descs, int32_t capacity, int32_t nsteps)
{
    const int idx = blockIdx.x * blockDim.x + threadIdx.x;
    const int k = idx / kMaxChunk, r = idx % kMaxChunk;
    if (k >= capacity || r >= nsteps) return;
    const InstDesc &d = descs[k];
    if (!d.active) return;
    const int t = d.t + r;
    if (t >= d.K) return;
    const float gamma = d.K > 1 ? d.gmin + (d.gmax - d.gmin) * ((float)t / (float)(d.K - 1)) : d.gmin;
    const float bc1 = -expm1f((float)(t + 1) * log1pf(d.b1 - 1.0f));
    const float bc2 = -expm1f((float)(t + 1) * log1pf(d.b2 - 1.0f));
    d.scal[r] = make_float4(gamma * (-2.0f * (float)d.a_ent), d.lr / bc1, rsqrtf(bc2), 0.0f);
}

void launch_prepare(const InstDesc *descs, int32_t capacity, int32_t nsteps, cudaStream_t st)
{
    const int total = capacity * kMaxChunk;
    prepare_kernel<<<(total + 127) / 128, 128, 0, st>>>(descs, capacity, nsteps);
}

// ---------------------------------------------------------------------------
// Projection rounding x = [p > 1/2] (Sec. 5) and exact integer costs.
// A slot is evaluated once per step count (skipped if already evaluated at t).
// ---------------------------------------------------------------------------
__device__ __forceinline__ bool needs_eval(const InstDesc &d) { return d.active && d.t != d.last_eval_t; }

__device__ __forceinline__ float state_value(const InstDesc &d, size_t e, int32_t prec)
{
    return prec == kFP32 ? reinterpret_cast<const float *>(d.X[d.t & 1])[e] : d.master[e];
}

// The evaluation runs on its own grid: blockIdx.y is the slot, blockIdx.x a
// chunk of `rows` consecutive rows of it (independent of the step kernel's
// tiles, which may be a few rows high).
//
// bits[i][w] bit b = (p[i][32w+b] > 1/2) for 32w+b < S; the first chunk of a
// slot zeroes its cost counters.
__global__ void eval_bits_kernel(const InstDesc *__restrict__ descs, int32_t rows, int32_t prec)
{
    const int lane = threadIdx.x & 31;
    const int warp = threadIdx.x >> 5;
    const int nwarps = blockDim.x >> 5;
    const InstDesc &d = descs[blockIdx.y];
    if (!needs_eval(d)) return;
    const int r0 = blockIdx.x * rows;
    if (r0 >= d.n) return;
    if (blockIdx.x == 0)
        for (int k = threadIdx.x; k < 3 * d.S_pad; k += blockDim.x) d.counts[k] = 0ULL;
    const int nr = min(rows, d.n - r0);
    const int pairs = nr * d.W;
    for (int pidx = warp; pidx < pairs; pidx += nwarps) {
        const int i = r0 + pidx / d.W;
        const int w = pidx % d.W;
        const int s = 32 * w + lane;
        const bool x = s < d.S && state_value(d, (size_t)i * d.S_pad + s, prec) > 0.5f;
        const unsigned word = __ballot_sync(0xffffffffu, x);
        if (lane == 0) d.bits[(size_t)i * d.W + w] = word;
    }
}

// Per replica: size = sum x_i, inside = #edges (i<j) with x_i x_j, cut = sum w_ij [x_i != x_j].
// Threads sharing a replica split the chunk's rows; each walks its rows'
// neighbour lists eight entries at a time with the index and bit-word loads
// of a batch in flight together. Partial counts are combined in shared
// memory, then added to the slot's counters. The neighbour lists of long rows
// are walked by blocks of their own, one per 32-entry segment (blocks past the
// slot's row chunks), so a hub does not hold up the evaluation; the counts are
// integers, so the split changes no result.
__global__ void eval_count_kernel(const InstDesc *__restrict__ descs, int32_t rows)
{
    extern __shared__ long long sh_cnt[];   // [3][S_pad32]
    const InstDesc &d = descs[blockIdx.y];
    if (!needs_eval(d) || d.dense_Abits) return;   // bitset slots are counted by eval_count_bits_kernel
    const int nchunks = (d.n + rows - 1) / rows;
    const bool seg_block = (int)blockIdx.x >= nchunks;
    int r0, row_end, ks0 = 0, ks1 = 0;
    if (!seg_block) {
        r0 = blockIdx.x * rows;
        row_end = min(r0 + rows, d.n);
    } else {
        const int q = blockIdx.x - nchunks;
        if (q >= d.nseg) return;   // block-uniform
        const int jl = d.seg_row[q];
        r0 = d.long_rows[jl];
        row_end = r0 + 1;
        ks0 = d.row_ptr[r0] + (q - d.seg_ptr[jl]) * kSegLen;
        ks1 = min(ks0 + kSegLen, d.row_ptr[r0 + 1]);
    }
    const int S32 = (d.S + 31) & ~31;
    for (int k = threadIdx.x; k < 3 * S32; k += blockDim.x) sh_cnt[k] = 0;
    __syncthreads();
    const int splits = max(1, (int)blockDim.x / S32);
    const int32_t *__restrict__ col = d.col;
    const int32_t *__restrict__ wts = d.w;
    const uint32_t *__restrict__ bits = d.bits;
    for (int base = threadIdx.x; base < splits * S32; base += blockDim.x) {
        const int s = base % S32;
        const int part = base / S32;
        if (s >= d.S) continue;
        const int w = s >> 5;
        const int b = s & 31;
        long long size = 0, inside = 0, cut = 0;
        for (int i = r0 + part; i < row_end; i += splits) {
            const unsigned xi = (bits[(size_t)i * d.W + w] >> b) & 1u;
            int kb = d.row_ptr[i], k1 = d.row_ptr[i + 1];
            if (seg_block) {
                kb = ks0;
                k1 = ks1;
            } else {
                size += xi;
                if (d.long_rows && k1 - kb > d.long_thresh) continue;   // walked by its segment blocks
            }
            for (int k = kb; k < k1; k += 8) {
                int j[8];
                unsigned word[8];
#pragma unroll
                for (int u = 0; u < 8; ++u) j[u] = k + u < k1 ? __ldg(col + k + u) : -1;
#pragma unroll
                for (int u = 0; u < 8; ++u) word[u] = j[u] > i ? __ldg(bits + (size_t)j[u] * d.W + w) : 0u;
#pragma unroll
                for (int u = 0; u < 8; ++u) {
                    if (j[u] <= i) continue;   // each undirected edge once (and past the row's end)
                    const unsigned xj = (word[u] >> b) & 1u;
                    inside += (long long)(xi & xj);
                    if (xi != xj) cut += wts ? (long long)__ldg(wts + k + u) : 1LL;
                }
            }
        }
        if (size) atomicAdd((unsigned long long *)&sh_cnt[s], (unsigned long long)size);
        if (inside) atomicAdd((unsigned long long *)&sh_cnt[S32 + s], (unsigned long long)inside);
        if (cut) atomicAdd((unsigned long long *)&sh_cnt[2 * S32 + s], (unsigned long long)cut);
    }
    __syncthreads();
    for (int s = threadIdx.x; s < d.S; s += blockDim.x) {
        if (sh_cnt[s]) atomicAdd(&d.counts[s], (unsigned long long)sh_cnt[s]);
        if (sh_cnt[S32 + s]) atomicAdd(&d.counts[d.S_pad + s], (unsigned long long)sh_cnt[S32 + s]);
        if (sh_cnt[2 * S32 + s]) atomicAdd(&d.counts[2 * d.S_pad + s], (unsigned long long)sh_cnt[2 * S32 + s]);
    }
}

// Slots with adjacency bitsets (unit-weight graphs on the tensor-core step):
// the rounded replicas transposed to node bitsets, xbits[s][k] bit b = x_{32k+b}
// of replica s. One warp per 32 x 32 block (32 nodes, 32 replicas): lane i
// holds the replica word of node 32k + i, and 32 ballots transpose it.
__global__ void eval_xbits_kernel(const InstDesc *__restrict__ descs)
{
    const InstDesc &d = descs[blockIdx.y];
    if (!needs_eval(d) || !d.dense_Abits) return;
    const int lane = threadIdx.x & 31;
    const int nw = d.n_pad >> 5;
    const int blk = blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5);
    if (blk >= nw * d.W) return;   // warp-uniform
    const int k = blk % nw, w = blk / nw;
    const int i = 32 * k + lane;
    const unsigned v = i < d.n ? d.bits[(size_t)i * d.W + w] : 0u;
    unsigned mine = 0;
#pragma unroll
    for (int b = 0; b < 32; ++b) {
        const unsigned m = __ballot_sync(0xffffffffu, (v >> b) & 1u);
        if (lane == b) mine = m;
    }
    d.dense_xbits[(size_t)(32 * w + lane) * nw + k] = mine;
}

// Exact costs by popcount, one warp per replica s (lanes over the 32-node
// words of a row): size = |X_s|; inside = sum over the selected nodes i of
// |N(i) & X_s|, halved (each edge is seen from both ends); unit-weight
// cut = sum of the selected nodes' degrees - 2 inside.
__global__ void eval_count_bits_kernel(const InstDesc *__restrict__ descs)
{
    const InstDesc &d = descs[blockIdx.y];
    if (!needs_eval(d) || !d.dense_Abits) return;
    const int lane = threadIdx.x & 31;
    const int s = blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5);
    if (s >= d.S) return;   // warp-uniform
    const int nw = d.n_pad >> 5;
    const uint32_t *xs = d.dense_xbits + (size_t)s * nw;
    long long size = 0, twice_inside = 0, degsum = 0;
    for (int kb = 0; kb < nw; kb += 32) {
        // this lane's word of X_s, then walk the selected nodes of every word of the batch
        const unsigned mine = kb + lane < nw ? xs[kb + lane] : 0u;
        size += __popc(mine);
        for (int kk = 0; kk < 32 && kb + kk < nw; ++kk) {
            unsigned sel = __shfl_sync(0xffffffffu, mine, kk);
            while (sel) {   // warp-uniform
                const int b = __ffs(sel) - 1;
                sel &= sel - 1;
                const int i = 32 * (kb + kk) + b;
                const uint32_t *arow = d.dense_Abits + (size_t)i * nw;
                for (int k = lane; k < nw; k += 32) twice_inside += __popc(arow[k] & xs[k]);
                if (lane == 0) degsum += d.row_ptr[i + 1] - d.row_ptr[i];
            }
        }
    }
#pragma unroll
    for (int off = 16; off > 0; off >>= 1) {
        size += __shfl_xor_sync(0xffffffffu, size, off);
        twice_inside += __shfl_xor_sync(0xffffffffu, twice_inside, off);
        degsum += __shfl_xor_sync(0xffffffffu, degsum, off);
    }
    if (lane == 0) {
        const long long inside = twice_inside / 2;
        d.counts[s] = (unsigned long long)size;
        d.counts[d.S_pad + s] = (unsigned long long)inside;
        d.counts[2 * d.S_pad + s] = (unsigned long long)(degsum - 2 * inside);
    }
}

// One warp per slot: objective, violation, feasibility, energy of every
// replica; best feasible replica (max objective, ties -> lowest s); history.
__global__ void eval_finalize_kernel(const InstDesc *__restrict__ descs_c, int32_t capacity)
{
    InstDesc *descs = const_cast<InstDesc *>(descs_c);
    const int lane = threadIdx.x & 31;
    const int slot = blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5);
    if (slot >= capacity) return;
    InstDesc &d = descs[slot];
    if (!needs_eval(d)) return;
    long long best_obj = 0;
    int best_s = -1;
    for (int s = lane; s < d.S; s += 32) {
        const long long size = (long long)d.counts[s];
        const long long inside = (long long)d.counts[d.S_pad + s];
        const long long cut = (long long)d.counts[2 * d.S_pad + s];
        long long obj, viol;
        double energy;
        if (d.kind == kMIS) {
            obj = size; viol = inside;
            energy = -(double)size + (double)d.lambda * (double)inside;
        } else if (d.kind == kMaxClique) {
            obj = size; viol = size * (size - 1) / 2 - inside;
            energy = -(double)size + (double)d.lambda * (double)viol;
        } else {
            obj = cut; viol = 0;
            energy = -(double)cut;
        }
        const bool feas = viol == 0;
        d.res_obj[s] = obj;
        d.res_viol[s] = viol;
        d.res_feas[s] = feas ? 1 : 0;
        d.res_energy[s] = energy;
        if (feas && (best_s < 0 || obj > best_obj)) { best_obj = obj; best_s = s; }
    }
    // warp argmax: larger objective wins, ties -> lower replica index
#pragma unroll
    for (int off = 16; off > 0; off >>= 1) {
        const long long o2 = __shfl_xor_sync(0xffffffffu, best_obj, off);
        const int s2 = __shfl_xor_sync(0xffffffffu, best_s, off);
        const bool take = s2 >= 0 && (best_s < 0 || o2 > best_obj || (o2 == best_obj && s2 < best_s));
        if (take) { best_obj = o2; best_s = s2; }
    }
    if (lane == 0) {
        const int count = d.res_meta[2];
        d.res_meta[0] = best_s;
        d.res_meta[1] = d.t;
        if (count < d.hist_cap) {
            d.hist_best[count] = best_s >= 0 ? best_obj : (long long)(-9223372036854775807LL - 1);
            d.hist_step[count] = d.t;
        }
        d.res_meta[2] = count + 1;
    }
}

// Bit-packed x of the best replica: one warp per 32 nodes, over the same
// (chunk, slot) grid as the counting kernels.
__global__ void eval_bestx_kernel(const InstDesc *__restrict__ descs, int32_t rows)
{
    const int lane = threadIdx.x & 31;
    const int warp = threadIdx.x >> 5;
    const InstDesc &d = descs[blockIdx.y];
    if (!needs_eval(d)) return;
    const int best_s = d.res_meta[0];
    const int w0 = blockIdx.x * (rows >> 5);
    const int nwords = (d.n + 31) >> 5;
    for (int word = w0 + warp; word < min(w0 + (rows >> 5), nwords); word += blockDim.x >> 5) {
        const int i = (word << 5) + lane;
        unsigned bit = 0;
        if (i < d.n && best_s >= 0) bit = (d.bits[(size_t)i * d.W + (best_s >> 5)] >> (best_s & 31)) & 1u;
        const unsigned packed = __ballot_sync(0xffffffffu, bit != 0);
        if (lane == 0) d.res_bestx[word] = packed;
    }
}

// The evaluation of step t is complete: later evaluations at the same t are skipped.
__global__ void eval_mark_kernel(InstDesc *__restrict__ descs, int32_t capacity)
{
    const int slot = blockIdx.x * blockDim.x + threadIdx.x;
    if (slot < capacity && needs_eval(descs[slot])) descs[slot].last_eval_t = descs[slot].t;
}

void launch_eval(const InstDesc *descs, int32_t capacity, int32_t n_max, int64_t total_rows, int32_t S_max_pad,
                 int32_t prec, bool dense, int32_t seg_max, cudaStream_t st)
{
    // rows per counting chunk: a multiple of 8, small enough for about four
    // waves of 256-thread blocks (8 per SM) over the whole run
    int sms = 152, dev = 0;
    if (cudaGetDevice(&dev) == cudaSuccess) cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    int rows = (int)std::min<int64_t>(256, std::max<int64_t>(8, total_rows / (32LL * sms)));
    rows = (rows + 7) & ~7;
    const dim3 grid(std::max(1, (n_max + rows - 1) / rows), capacity);
    eval_bits_kernel<<<grid, 256, 0, st>>>(descs, rows, prec);
    const int S32 = (S_max_pad + 31) & ~31;
    const dim3 grid_c(grid.x + (unsigned)seg_max, capacity);   // row chunks, then long-row segments
    eval_count_kernel<<<grid_c, 256, 3 * S32 * sizeof(long long), st>>>(descs, rows);
    if (dense) {   // unit-weight slots of the tensor-core step: costs by popcount over bitsets
        const int nw = (n_max + 127) / 128 * 4;   // 32-node words of the largest n_pad
        const int W = S32 / 32;
        eval_xbits_kernel<<<dim3((nw * W + 7) / 8, capacity), 256, 0, st>>>(descs);
        eval_count_bits_kernel<<<dim3((S32 + 7) / 8, capacity), 256, 0, st>>>(descs);
    }
    eval_finalize_kernel<<<(capacity + 7) / 8, 256, 0, st>>>(descs, capacity);
    // best x: 1024 rows (32 words) per block
    const dim3 grid_b(std::max(1, (n_max + 1023) / 1024), capacity);
    eval_bestx_kernel<<<grid_b, 256, 0, st>>>(descs, 1024);
    eval_mark_kernel<<<(capacity + 127) / 128, 128, 0, st>>>(const_cast<InstDesc *>(descs), capacity);
}

// ---------------------------------------------------------------------------
// State export/import between the padded device layout and dense FP32 [n][S].
// which: 0 = p (X or master), 1 = m, 2 = v.
// ---------------------------------------------------------------------------
__global__ void pack_state_kernel(const InstDesc *__restrict__ descs, int32_t slot, int32_t prec, int32_t which,
                                  float *__restrict__ dst)
{
    const InstDesc &d = descs[slot];
    const long long total = (long long)d.n * d.S;
    for (long long idx = blockIdx.x * (long long)blockDim.x + threadIdx.x; idx < total;
         idx += (long long)gridDim.x * blockDim.x) {
        const int i = (int)(idx / d.S), s = (int)(idx % d.S);
        const size_t e = (size_t)i * d.S_pad + s;
        float val;
        if (which == 0) val = state_value(d, e, prec);
        else {
            const void *src = which == 1 ? d.m : d.v;
            val = prec == kFP32 ? reinterpret_cast<const float *>(src)[e]
                                : __bfloat162float(reinterpret_cast<const __nv_bfloat16 *>(src)[e]);
        }
        dst[idx] = val;
    }
}

void launch_pack_state(const InstDesc *descs, int32_t slot, int32_t n, int32_t S, int32_t S_pad, int32_t prec,
                       int32_t which, float *dst, cudaStream_t st)
{
    (void)S_pad;
    const long long total = (long long)n * S;
    const int grid = (int)((total + 255) / 256 < 65535 ? (total + 255) / 256 : 65535);
    pack_state_kernel<<<grid > 0 ? grid : 1, 256, 0, st>>>(descs, slot, prec, which, dst);
}

// X, m, v are dense FP32 [n][S] device arrays; the state buffer for step t is
// X[t & 1]; padded replicas (S <= s < S_pad) are left as they are.
__global__ void unpack_state_kernel(const InstDesc *__restrict__ descs, int32_t slot, int32_t prec,
                                    const float *__restrict__ X, const float *__restrict__ m,
                                    const float *__restrict__ v, int32_t t)
{
    const InstDesc &d = descs[slot];
    const long long total = (long long)d.n * d.S;
    for (long long idx = blockIdx.x * (long long)blockDim.x + threadIdx.x; idx < total;
         idx += (long long)gridDim.x * blockDim.x) {
        const int i = (int)(idx / d.S), s = (int)(idx % d.S);
        const size_t e = (size_t)i * d.S_pad + s;
        if (prec == kFP32) {
            reinterpret_cast<float *>(d.X[t & 1])[e] = X[idx];
            reinterpret_cast<float *>(d.m)[e] = m[idx];
            reinterpret_cast<float *>(d.v)[e] = v[idx];
        } else {
            d.master[e] = X[idx];
            reinterpret_cast<__nv_bfloat16 *>(d.X[t & 1])[e] = __float2bfloat16_rn(X[idx]);
            reinterpret_cast<__nv_bfloat16 *>(d.m)[e] = __float2bfloat16_rn(m[idx]);
            reinterpret_cast<__nv_bfloat16 *>(d.v)[e] = __float2bfloat16_rn(v[idx]);
        }
    }
}

void launch_unpack_state(const InstDesc *descs, int32_t slot, int32_t n, int32_t S, int32_t S_pad, int32_t prec,
                         const float *X, const float *m, const float *v, int32_t t, cudaStream_t st)
{
    (void)S_pad;
    const long long total = (long long)n * S;
    const int grid = (int)((total + 255) / 256 < 65535 ? (total + 255) / 256 : 65535);
    unpack_state_kernel<<<grid > 0 ? grid : 1, 256, 0, st>>>(descs, slot, prec, X, m, v, t);
}

__global__ void copy_grad_kernel(int32_t n, int32_t S, int32_t S_pad, const float *__restrict__ src,
                                 float *__restrict__ dst)
{
    const long long total = (long long)n * S;
    for (long long idx = blockIdx.x * (long long)blockDim.x + threadIdx.x; idx < total;
         idx += (long long)gridDim.x * blockDim.x) {
        const int i = (int)(idx / S), s = (int)(idx % S);
        dst[idx] = src[(size_t)i * S_pad + s];
    }
}

void launch_copy_grad(const InstDesc *descs, int32_t slot, int32_t n, int32_t S, int32_t S_pad, const float *src,
                      float *dst, cudaStream_t st)
{
    (void)descs; (void)slot;
    const long long total = (long long)n * S;
    const int grid = (int)((total + 255) / 256 < 65535 ? (total + 255) / 256 : 65535);
    copy_grad_kernel<<<grid > 0 ? grid : 1, 256, 0, st>>>(n, S, S_pad, src, dst);
}

}  // namespace qqa
