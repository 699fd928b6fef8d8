// step_dense.cu -- the product of the PQQA step on the 5th-generation tensor
// cores, for dense graphs (FP32 runs, and BF16 runs, whose planes come from
// the FP32 master).
//
// The sparse product of the step, Y[i][s] = sum_j A_ij p^t[j][s] (Eqs. 22, 24,
// 26), is a dense contraction when the graph is dense (ER with p = 0.15 has
// about 112 neighbours per 750 nodes). Here it runs as a GEMM on tcgen05:
//   - A is kept as an fp16 adjacency [n_pad][n_pad] (0/1 or small integer
//     weights, exact in fp16), zero padded to a multiple of 128;
//   - p^t is kept, besides its FP32 copy, as two fp16 planes hi = fp16(p) and
//     lo = fp16(p - hi), stored transposed ([s][j]); hi + lo carries about 22
//     significant bits, and D = A.hi + A.lo is accumulated in FP32 in tensor
//     memory (every product is exact), so Y matches the FP32 gather to the
//     rounding of an FP32 sum;
//   - one CTA owns 128 rows of one instance: one thread streams 64-wide K
//     chunks of A and of both planes into shared memory with TMA (128-byte
//     swizzle, 4 stages - 2 at N = 256 - mbarrier completion, bounded waits),
//     another issues tcgen05.mma (M = 128, N = dense_N, K = 16) into a TMEM
//     accumulator as the chunks land, and four warps read the accumulator
//     with tcgen05.ld and store Y [n][S_pad] (FP32).
// The rest of the step (gradient, statistics, AdamW, noise, clamp, and the
// next step's planes) is the update kernel of step_dense_update.cu, which
// runs on every SM over 32-row tiles.
#include <cuda.h>
#include <cuda_fp16.h>

#include "step_impl.cuh"

namespace qqa {

namespace {

// pipeline depth: four stages up to N = 128 (48 KB each), two at N = 256 (80 KB each)
__host__ __device__ constexpr int dense_stages(int N) { return N >= 256 ? 2 : 4; }
constexpr int kGemmThreads = 6 * 32;   // warps 0-3: accumulator -> Y; warp 4: TMA loads; warp 5: MMAs

__device__ __forceinline__ uint64_t umma_desc_sw128(uint32_t saddr)
{
    // K-major operand, 128-byte swizzle: start address >> 4, leading byte
    // offset (unused for this layout) 1, stride byte offset 1024 >> 4 (eight
    // 128-byte rows), descriptor version 1, layout type 2 (128B swizzle)
    return (uint64_t)((saddr >> 4) & 0x3FFF) | ((uint64_t)1 << 16) | ((uint64_t)64 << 32) | ((uint64_t)1 << 46) |
           ((uint64_t)2 << 61);
}

__device__ __forceinline__ void tma_load_2d(uint32_t dst, const void *tmap, int x, int y, uint32_t mbar)
{
    asm volatile(
        "cp.async.bulk.tensor.2d.shared::cluster.global.tile.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3}], [%4];" ::"r"(
            dst),
        "l"(tmap), "r"(x), "r"(y), "r"(mbar)
        : "memory");
}

__device__ __forceinline__ void mma_f16(uint32_t tmem_d, uint64_t a, uint64_t b, uint32_t idesc, uint32_t accumulate)
{
    asm volatile("{\n\t.reg .pred p;\n\tsetp.ne.b32 p, %4, 0;\n\t"
                 "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n\t}" ::"r"(tmem_d),
                 "l"(a), "l"(b), "r"(idesc), "r"(accumulate)
                 : "memory");
}

__device__ __forceinline__ void mma_commit(uint32_t mbar)
{
    asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(mbar) : "memory");
}

__device__ __forceinline__ void tmem_ld16(uint32_t taddr, uint32_t (&r)[16])
{
    asm volatile("tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15}, [%16];"
                 : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]),
                   "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15])
                 : "r"(taddr));
    asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
}

__device__ __forceinline__ bool mbar_wait_limit(uint32_t mbar, uint32_t parity)
{
    const long long start = clock64();
    while (true) {
        uint32_t ok;
        asm volatile("{\n\t.reg .pred p;\n\tmbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\tselp.u32 %0, 1, 0, p;\n\t}"
                     : "=r"(ok)
                     : "r"(mbar), "r"(parity)
                     : "memory");
        if (ok) return true;
        if (clock64() - start > (1LL << 31)) return false;   // ~1 s
    }
}

}  // namespace

// ---------------------------------------------------------------------------
// Product kernel: Y = A p^t for 128 rows of one instance per tile. Warp 4's
// first lane streams 64-wide K chunks of the fp16 adjacency and of both fp16
// planes of p^t with TMA, warp 5's first lane issues tcgen05.mma on them (M =
// 128, N = the MMA width, K = 16; hi and lo accumulate into the same FP32
// accumulator); warps 0-3 read
// the accumulator (TMEM lane = row, column = replica) and store Y[row][s] for
// the update kernel. N = MMA width (64, 128 or 256 replicas). The loads and
// the MMAs are issued by two different warps, so the tensor cores take each
// chunk as soon as it lands while the loads run up to four stages ahead.
// ---------------------------------------------------------------------------
template <int N>
__global__ void __launch_bounds__(kGemmThreads, 1) qqa_dense_gemm_kernel(const InstDesc *__restrict__ descs,
                                                                         const Tile *__restrict__ tiles,
                                                                         const int32_t *__restrict__ num_tiles_p,
                                                                         RunStatus *__restrict__ status, int32_t r)
{
    constexpr int A_BYTES = 128 * 128;       // 128 rows x 64 fp16
    constexpr int B_BYTES = N * 128;         // N rows x 64 fp16
    constexpr int STAGE = A_BYTES + 2 * B_BYTES;
    constexpr int kDenseStages = dense_stages(N);
    extern __shared__ __align__(1024) unsigned char dsm_raw[];
    unsigned char *base = (unsigned char *)(((uintptr_t)dsm_raw + 1023) & ~(uintptr_t)1023);
    unsigned char *stages = base;
    uint64_t *mb_full = reinterpret_cast<uint64_t *>(base + kDenseStages * STAGE);
    uint64_t *mb_empty = mb_full + kDenseStages;
    uint64_t *mb_acc = mb_empty + kDenseStages;
    uint32_t *tmem_slot = reinterpret_cast<uint32_t *>(mb_acc + 1);

    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int num_tiles = *num_tiles_p;

    if (threadIdx.x == 0) {
        for (int k = 0; k < kDenseStages; ++k) {
            asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(smem_addr(mb_full + k)) : "memory");
            asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(smem_addr(mb_empty + k)) : "memory");
        }
        asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(smem_addr(mb_acc)) : "memory");
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    if (warp == 0) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_addr(tmem_slot)),
                     "n"(N)
                     : "memory");
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
    }
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncthreads();
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    const uint32_t tmem = *tmem_slot;

    uint32_t chunk_base = 0;   // K chunks this CTA has streamed so far (producer and MMA warps)
    uint32_t tiles_done = 0;   // accumulator phases completed (all threads)
    bool failed = false;

    for (int tile = blockIdx.x; tile < num_tiles && !failed; tile += gridDim.x) {
        const Tile tl = tiles[tile];
        const InstDesc *__restrict__ d = descs + tl.slot;
        const int t = d->t + r;
        if (t >= d->K) continue;   // block-uniform
        const int n = d->n, n_pad = d->n_pad, nK = n_pad / 64;

        if (warp == 4) {
            if (lane == 0) {
                // ---------------- producer: TMA loads of the K chunks ----------------
                const CUtensorMap *tm = reinterpret_cast<const CUtensorMap *>(d->dense_tmaps);
                const CUtensorMap *tmA = tm, *tmH = tm + 1 + 2 * (t & 1), *tmL = tmH + 1;
                asm volatile("fence.proxy.tensormap::generic.acquire.gpu [%0], 128;" ::"l"(tmA) : "memory");
                asm volatile("fence.proxy.tensormap::generic.acquire.gpu [%0], 128;" ::"l"(tmH) : "memory");
                asm volatile("fence.proxy.tensormap::generic.acquire.gpu [%0], 128;" ::"l"(tmL) : "memory");
                for (int kc = 0; kc < nK; ++kc) {
                    const uint32_t f = chunk_base + kc;
                    const int st = f % kDenseStages;
                    // the stage is free once the MMAs that read it last have completed
                    if (f >= kDenseStages && !mbar_wait_limit(smem_addr(mb_empty + st), ((f / kDenseStages) - 1) & 1)) {
                        atomicAdd(&status->timeouts, 1ULL);
                        break;
                    }
                    unsigned char *sp = stages + st * STAGE;
                    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_addr(mb_full + st)),
                                 "r"(STAGE)
                                 : "memory");
                    tma_load_2d(smem_addr(sp), tmA, 64 * kc, tl.row0, smem_addr(mb_full + st));
                    tma_load_2d(smem_addr(sp + A_BYTES), tmH, 64 * kc, 0, smem_addr(mb_full + st));
                    tma_load_2d(smem_addr(sp + A_BYTES + B_BYTES), tmL, 64 * kc, 0, smem_addr(mb_full + st));
                }
            }
            __syncwarp();
            chunk_base += nK;
        } else if (warp == 5) {
            if (lane == 0) {
                // ---------------- MMA issuer: one chunk after the other as they land ----------------
                const uint32_t idesc = (1u << 4) | ((uint32_t)(N >> 3) << 17) | ((uint32_t)(128 >> 4) << 24);
                bool ok = true;
                for (int kc = 0; kc < nK; ++kc) {
                    const uint32_t c = chunk_base + kc;
                    const int st = c % kDenseStages;
                    ok = mbar_wait_limit(smem_addr(mb_full + st), (c / kDenseStages) & 1);
                    if (!ok) break;
                    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
                    const uint32_t sa = smem_addr(stages + st * STAGE);
#pragma unroll
                    for (int ks = 0; ks < 4; ++ks) {
                        const uint64_t ad = umma_desc_sw128(sa + ks * 32);
                        const uint64_t bh = umma_desc_sw128(sa + A_BYTES + ks * 32);
                        const uint64_t bl = umma_desc_sw128(sa + A_BYTES + B_BYTES + ks * 32);
                        mma_f16(tmem, ad, bh, idesc, (kc > 0 || ks > 0) ? 1u : 0u);
                        mma_f16(tmem, ad, bl, idesc, 1u);
                    }
                    mma_commit(smem_addr(mb_empty + st));   // stage free once these MMAs are done
                }
                if (ok) mma_commit(smem_addr(mb_acc));     // accumulator complete
                else atomicAdd(&status->timeouts, 1ULL);
            }
            __syncwarp();
            chunk_base += nK;
        } else {
            // ---------------- warps 0-3: accumulator -> Y ----------------
            const bool acc_ok = mbar_wait_limit(smem_addr(mb_acc), tiles_done & 1);
            asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
            if (!acc_ok) {
                if (threadIdx.x == 0) atomicAdd(&status->timeouts, 1ULL);
                failed = true;
            } else {
                const int row = tl.row0 + 32 * warp + lane;   // TMEM lane = row of the tile
                const int S_pad = d->S_pad;
                float *yrow = d->dense_Y + (size_t)row * S_pad;
#pragma unroll 1
                for (int c16 = 0; c16 < N && c16 < S_pad; c16 += 16) {
                    uint32_t yr[16];
                    tmem_ld16(tmem + ((uint32_t)(32 * warp) << 16) + (uint32_t)c16, yr);
                    if (row < n) {
#pragma unroll
                        for (int e = 0; e < 16; e += 4)
                            if (c16 + e < S_pad)
                                *reinterpret_cast<float4 *>(yrow + c16 + e) =
                                    make_float4(__uint_as_float(yr[e]), __uint_as_float(yr[e + 1]),
                                                __uint_as_float(yr[e + 2]), __uint_as_float(yr[e + 3]));
                    }
                }
            }
            asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
        }
        ++tiles_done;
        failed = __syncthreads_or(failed);   // the accumulator is reused by the next tile
        asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    }
    __syncthreads();
    if (warp == 0) {
        asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "n"(N) : "memory");
    }
}

using StepFn = void (*)(const InstDesc *, const Tile *, const int32_t *, RunStatus *, int32_t);

StepFn dense_gemm_kernel(int N)
{
    if (N == 64) return qqa_dense_gemm_kernel<64>;
    if (N == 128) return qqa_dense_gemm_kernel<128>;
    if (N == 256) return qqa_dense_gemm_kernel<256>;
    return nullptr;
}

int dense_gemm_threads() { return kGemmThreads; }

int dense_smem_bytes(int N)
{
    const int stage = 128 * 128 + 2 * N * 128;
    const int ns = dense_stages(N);
    return 1024 + ns * stage + (2 * ns + 1) * 8 + 16 + 64;
}

// ---------------------------------------------------------------------------
// Dense data of a slot: the fp16 adjacency (zeroed by the host first) and the
// fp16 planes of the state p^t (buffer t & 1).
// ---------------------------------------------------------------------------
__global__ void dense_adjacency_kernel(const InstDesc *__restrict__ descs, int32_t slot)
{
    const InstDesc &d = descs[slot];
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < d.n; i += gridDim.x * blockDim.x) {
        __half *row = reinterpret_cast<__half *>(d.dense_A) + (size_t)i * d.n_pad;
        uint32_t *brow = d.dense_Abits ? d.dense_Abits + (size_t)i * (d.n_pad / 32) : nullptr;
        for (int k = d.row_ptr[i]; k < d.row_ptr[i + 1]; ++k) {
            const int j = d.col[k];
            row[j] = __float2half_rn(d.w ? (float)d.w[k] : 1.0f);
            if (brow) brow[j >> 5] |= 1u << (j & 31);   // this thread owns row i
        }
    }
}

__global__ void dense_planes_kernel(const InstDesc *__restrict__ descs, int32_t slot)
{
    const InstDesc &d = descs[slot];
    const int b = d.t & 1;
    const float *X = d.master ? d.master : reinterpret_cast<const float *>(d.X[b]);   // p^t in FP32
    __half *hi = reinterpret_cast<__half *>(d.dense_XT) + (size_t)b * 2 * d.dense_N * d.n_pad;
    __half *lo = hi + (size_t)d.dense_N * d.n_pad;
    const long long total = (long long)d.n * d.S_pad;
    for (long long idx = blockIdx.x * (long long)blockDim.x + threadIdx.x; idx < total;
         idx += (long long)gridDim.x * blockDim.x) {
        const int j = (int)(idx % d.n), s = (int)(idx / d.n);   // consecutive threads: consecutive j
        const float x = X[(size_t)j * d.S_pad + s];
        const __half h = __float2half_rn(x);
        hi[(size_t)s * d.n_pad + j] = h;
        lo[(size_t)s * d.n_pad + j] = __float2half_rn(x - __half2float(h));
    }
}

void launch_dense_adjacency(const InstDesc *descs, int32_t slot, int32_t n, cudaStream_t st)
{
    dense_adjacency_kernel<<<(n + 127) / 128, 128, 0, st>>>(descs, slot);
}

void launch_dense_planes(const InstDesc *descs, int32_t slot, int32_t n, int32_t S_pad, cudaStream_t st)
{
    const long long total = (long long)n * S_pad;
    const int grid = (int)((total + 255) / 256 < 65535 ? (total + 255) / 256 : 65535);
    dense_planes_kernel<<<grid > 0 ? grid : 1, 256, 0, st>>>(descs, slot);
}

}  // namespace qqa
