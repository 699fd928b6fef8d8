// qqa_internal.cuh -- device-side data layout and helpers of libqqa (sm_103a).
//
// One InstDesc per slot lives in device memory; every kernel reads the
// instance it works on from it. Replica state is node-major [n][S_pad] with
// S_pad = S rounded up to one 16-byte vector (4 FP32 or 8 BF16 replicas), so
// every row starts 16-byte aligned and a group of lanes reads a row with
// 128-bit coalesced loads.
#pragma once

#include <cuda_bf16.h>
#include <cuda_runtime.h>
#include <stddef.h>
#include <stdint.h>

namespace qqa {

enum Kind : int32_t { kMIS = 0, kMaxCut = 1, kMaxClique = 2 };
enum Prec : int32_t { kFP32 = 0, kBF16 = 1 };

struct __align__(16) InstDesc {
    // graph (device CSR, owned by the problem)
    const int32_t *row_ptr;
    const int32_t *col;
    const int32_t *w;            // edge weights (max-cut) or nullptr = unit
    // state
    void *X[2];                  // ping-pong p^t / p^{t+1}: float or bf16 [n][S_pad]
    float *master;               // BF16 runs: FP32 master copy of p [n][S_pad]; FP32 runs: nullptr
    void *m;                     // AdamW first moment  (float or bf16) [n][S_pad]
    void *v;                     // AdamW second moment (float or bf16) [n][S_pad]
    float *colsum;               // max-clique: column sums sum_i p_is of the current state [S_pad]
    float *grad_dbg;             // optional gradient dump [n][S_pad] (debug step only)
    // evaluation scratch and results
    uint32_t *bits;              // rounded replicas [n][W] (bit s%32 of word s/32)
    unsigned long long *counts;  // per replica: size, inside edges, cut weight (as two's complement) [3][S_pad]
    long long *res_obj;          // [S_pad]
    long long *res_viol;         // [S_pad]
    uint8_t *res_feas;           // [S_pad]
    double *res_energy;          // [S_pad]
    int32_t *res_meta;           // [0] best_s, [1] step of the evaluation, [2] evaluations done
    uint32_t *res_bestx;         // [ceil(n/32)]
    long long *hist_best;        // [hist_cap]
    int32_t *hist_step;          // [hist_cap]
    float4 *scal;                // per-step scalars of the current chunk [kMaxChunk]: x = gamma_t * (-2a),
                                 // y = lr / (1 - b1^(t+1)), z = 1 / sqrt(1 - b2^(t+1))
    // dense tensor-core path (dense graphs); null otherwise
    uint16_t *dense_A;           // fp16 adjacency [n_pad][n_pad], zero padded
    uint16_t *dense_XT;          // fp16 state planes [2 buffers][2 (hi, lo)][dense_N][n_pad]: p^t[j][s] at [s][j]
    const void *dense_tmaps;     // 5 TMA tensor maps: adjacency, then planes (buffer 0 hi, lo, buffer 1 hi, lo)
    uint32_t *dense_Abits;       // unit-weight graphs: adjacency bitsets [n_pad][n_pad / 32] (bit j of row i = A_ij)
    uint32_t *dense_xbits;       // rounded replicas as node bitsets [S rounded to 32][n_pad / 32]
    float *dense_Y;              // the tensor cores' product A.p^t [n][S_pad] (FP32), read by the update
    const void *pad_ptr2;
    int32_t n_pad, dense_N;
    int32_t long_thresh;         // rows with more neighbours than this are long (INT32_MAX: none)
    int32_t hub_active;          // 1: the step kernels leave long rows to the segment work items
    // long rows: their neighbour lists are summed in segments of kSegLen entries
    // by separate work items (tables owned by the problem; the evaluation splits
    // them the same way; partial sums and arrival counters owned by the slot,
    // present when hub_active)
    const int32_t *long_rows;    // [nlong] node index of each long row
    const int32_t *seg_ptr;      // [nlong + 1] first segment of each long row
    const int32_t *seg_row;      // [nseg] long row (index into long_rows) of each segment
    float *seg_part;             // [nseg][S_pad] FP32 partial neighbour sums of the current step
    uint32_t *seg_cnt;           // [nlong] segments of the current step done (reset to 0 by the last one)
    int32_t nlong, nseg;
    // sizes
    int32_t n, S, S_pad, W;
    int32_t kind, a_ent, t, K;
    int32_t active, hist_cap, last_eval_t, pad0;
    // hyper-parameters
    float lr, wd, b1, b2;
    float adam_eps, gmin, gmax, alpha;
    float comm_eps, noise_scale, lambda, decay;   // decay = 1 - lr * weight_decay
    uint32_t seed_lo, seed_hi, pad2, pad3;
};

// Device status word of a run.
struct RunStatus {
    unsigned long long nonfinite;   // count of non-finite gradient / state values seen
    unsigned long long timeouts;    // bounded mbarrier waits that ran out (staged, pipelined, tensor-core kernels)
};

// Longest run of steps launched back to back (one chunk); the per-step scalar
// table of each slot holds this many entries.
constexpr int kMaxChunk = 64;

// Tiles: (slot, first row). A block processes one tile at a time. The
// long-row work items use the same record with row0 = the segment index.
struct Tile {
    int32_t slot;
    int32_t row0;
};

// Neighbours per segment of a long row.
constexpr int kSegLen = 32;

// A tile record with row0 < 0 stands for segment work items of long rows (the
// pipelined kernel's list): segments -row0 - 1, ..., one per lane group.
__host__ __device__ __forceinline__ int32_t seg_item_first(int32_t row0) { return -row0 - 1; }

// ---------------------------------------------------------------------------
// Philox4x32-10 counter-based generator (Salmon, Moraes, Dror, Shaw, SC'11):
// ten rounds of two 32x32->64 multiplications with the published multipliers,
// xor with the round key, and a Weyl-sequence key schedule.
// ---------------------------------------------------------------------------
struct U4 {
    uint32_t x, y, z, w;
};

__device__ __forceinline__ U4 philox10(U4 c, uint32_t k0, uint32_t k1)
{
#pragma unroll
    for (int round = 0; round < 10; ++round) {
        const uint64_t p0 = (uint64_t)0xD2511F53u * c.x;   // one widening multiply gives hi and lo
        const uint64_t p1 = (uint64_t)0xCD9E8D57u * c.z;
        const uint32_t lo0 = (uint32_t)p0, hi0 = (uint32_t)(p0 >> 32);
        const uint32_t lo1 = (uint32_t)p1, hi1 = (uint32_t)(p1 >> 32);
        c = U4{hi1 ^ c.y ^ k0, lo1, hi0 ^ c.w ^ k1, lo0};
        k0 += 0x9E3779B9u;
        k1 += 0xBB67AE85u;
    }
    return c;
}

// uniform in (0, 1]: the top 24 bits plus one, scaled by 2^-24 (exact in FP32)
__device__ __forceinline__ float bits_to_unit(uint32_t r)
{
    return (float)((r >> 8) + 1u) * 5.9604644775390625e-8f;
}

// Single-instruction approximations of the PTX ISA (flush-to-zero forms: the
// step's values are never subnormal, and these skip the subnormal handling):
// relative errors of a few ulp, far inside the single-step tolerance.
__device__ __forceinline__ float rsqrt_ftz(float x)
{
    float y;
    asm("rsqrt.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
    return y;
}

__device__ __forceinline__ float rcp_ftz(float x)
{
    float y;
    asm("rcp.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
    return y;
}

// sqrt(x) for x >= 0 (0 -> 0).
__device__ __forceinline__ float sqrt_nonneg(float x)
{
    float y;
    asm("sqrt.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
    return y;
}

__device__ __forceinline__ float log2_ftz(float x)
{
    float y;
    asm("lg2.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
    return y;
}

// -2 ln(u) for u = ((r >> 8) + 1) 2^-24 in (0, 1], the Box-Muller radius squared.
// delta = 1 - u = ((~r) >> 8) 2^-24 and u = 1 - delta are exact. Away from u = 1
// the hardware log2 is accurate relative to the result; close to u = 1 its
// absolute error is not, so for delta < 2^-10 the Taylor series
// -2 ln(1 - delta) = 2 delta + delta^2 + (2/3) delta^3 + ... is cut after two
// terms (relative error below delta^2 / 3 < 3.2e-7).
__device__ __forceinline__ float neg2_log_unit(uint32_t r)
{
    const float delta = (float)((~r) >> 8) * 5.9604644775390625e-8f;
    const float series = fmaf(delta, delta, delta + delta);
    const float via_log2 = -1.38629436111989061883f * log2_ftz(1.0f - delta);   // -2 ln 2 log2(u)
    return delta < 9.765625e-4f ? series : via_log2;
}

// NQ independent Philox4x32-10 streams in lockstep: one key schedule for all
// of them, and NQ-fold instruction-level parallelism.
template <int NQ>
__device__ __forceinline__ void philox10_multi(U4 (&c)[NQ], uint32_t k0, uint32_t k1)
{
#pragma unroll
    for (int round = 0; round < 10; ++round) {
#pragma unroll
        for (int j = 0; j < NQ; ++j) {
            const uint64_t p0 = (uint64_t)0xD2511F53u * c[j].x;
            const uint64_t p1 = (uint64_t)0xCD9E8D57u * c[j].z;
            c[j] = U4{(uint32_t)(p1 >> 32) ^ c[j].y ^ k0, (uint32_t)p1, (uint32_t)(p0 >> 32) ^ c[j].w ^ k1, (uint32_t)p0};
        }
        k0 += 0x9E3779B9u;
        k1 += 0xBB67AE85u;
    }
}

// Box-Muller pair from the uniform words (ra, rb): radius sqrt(-2 ln u1) with
// u1 from ra, angle 2 pi u2 with u2 from rb. The angle is taken as
// 2 pi (u2 - 1/2) = ((rb >> 8) - (2^23 - 1)) * (2 pi 2^-24) - exact in FP32 up to
// the one rounding of the product, so the hardware sine/cosine see (-pi, pi];
// the sign flip restores cos/sin(2 pi u2).
__device__ __forceinline__ void box_muller(uint32_t ra, uint32_t rb, float &z0, float &z1)
{
    const float rad = sqrt_nonneg(neg2_log_unit(ra));
    const float ang = (float)((int32_t)(rb >> 8) - 8388607) * 0x1.921FB6p-22f;   // fl(2 pi) * 2^-24
    float sn, cs;
    __sincosf(ang, &sn, &cs);
    z0 = -rad * cs;
    z1 = -rad * sn;
}

// Standard normals for the NQ replica quads q[j] of node i at step t (stream
// tag 1): out[4j..4j+3] are replicas 4 q[j] .. 4 q[j] + 3, Box-Muller on the
// uniform pairs (r0, r1) and (r2, r3) of each quad's Philox block.
template <int NQ>
__device__ __forceinline__ void gauss_quads(uint32_t seed_lo, uint32_t seed_hi, uint32_t i, const uint32_t (&q)[NQ],
                                            uint32_t t, float *out)
{
    U4 c[NQ];
#pragma unroll
    for (int j = 0; j < NQ; ++j) c[j] = U4{i, q[j], t, 1u};
    philox10_multi<NQ>(c, seed_lo, seed_hi);
#pragma unroll
    for (int j = 0; j < NQ; ++j) {
        box_muller(c[j].x, c[j].y, out[4 * j], out[4 * j + 1]);
        box_muller(c[j].z, c[j].w, out[4 * j + 2], out[4 * j + 3]);
    }
}

// Four standard normals for replicas 4q..4q+3 of node i at step t.
__device__ __forceinline__ void gauss4(uint32_t seed_lo, uint32_t seed_hi, uint32_t i, uint32_t q, uint32_t t,
                                       float out[4])
{
    const uint32_t qs[1] = {q};
    gauss_quads<1>(seed_lo, seed_hi, i, qs, t, out);
}

// Four uniforms for the initial state (stream tag 0, step 0).
__device__ __forceinline__ void unif4(uint32_t seed_lo, uint32_t seed_hi, uint32_t i, uint32_t q, float out[4])
{
    const U4 r = philox10(U4{i, q, 0u, 0u}, seed_lo, seed_hi);
    out[0] = bits_to_unit(r.x);
    out[1] = bits_to_unit(r.y);
    out[2] = bits_to_unit(r.z);
    out[3] = bits_to_unit(r.w);
}

// ---------------------------------------------------------------------------
// L2 cache policies (createpolicy) and the hinted 16-byte accesses that use
// them: state streamed once per step is marked evict-first, the state vector
// the next step gathers from is marked evict-last.
// ---------------------------------------------------------------------------
struct L2Policies {
    uint64_t stream;   // read or written once per step
    uint64_t keep;     // gathered again (p^t, p^{t+1})
};

__device__ __forceinline__ L2Policies make_l2_policies(bool hints)
{
    uint64_t first, last, normal;
    asm volatile("createpolicy.fractional.L2::evict_first.b64 %0, 1.0;" : "=l"(first));
    asm volatile("createpolicy.fractional.L2::evict_last.b64 %0, 1.0;" : "=l"(last));
    asm volatile("createpolicy.fractional.L2::evict_normal.b64 %0, 1.0;" : "=l"(normal));
    return hints ? L2Policies{first, last} : L2Policies{normal, normal};
}

__device__ __forceinline__ uint4 ld_nc_hint(const void *p, uint64_t pol)
{
    uint4 v;
    asm("ld.global.nc.L2::cache_hint.v4.u32 {%0, %1, %2, %3}, [%4], %5;"
        : "=r"(v.x), "=r"(v.y), "=r"(v.z), "=r"(v.w)
        : "l"(p), "l"(pol));
    return v;
}

__device__ __forceinline__ void st_hint(void *p, uint4 v, uint64_t pol)
{
    asm volatile("st.global.L2::cache_hint.v4.b32 [%0], {%1, %2, %3, %4}, %5;" ::"l"(p), "r"(v.x), "r"(v.y),
                 "r"(v.z), "r"(v.w), "l"(pol)
                 : "memory");
}

// ---------------------------------------------------------------------------
// 16-byte vectors of replicas: 4 FP32 or 8 BF16 values.
// ---------------------------------------------------------------------------
template <typename T>
struct VecT;

template <>
struct VecT<float> {
    static constexpr int N = 4;
    __device__ __forceinline__ static void load(const float *p, float out[4])
    {
        const float4 a = *reinterpret_cast<const float4 *>(p);
        out[0] = a.x; out[1] = a.y; out[2] = a.z; out[3] = a.w;
    }
    __device__ __forceinline__ static void load_ro(const float *p, float out[4])
    {
        const float4 a = __ldg(reinterpret_cast<const float4 *>(p));
        out[0] = a.x; out[1] = a.y; out[2] = a.z; out[3] = a.w;
    }
    __device__ __forceinline__ static void store(float *p, const float in[4])
    {
        *reinterpret_cast<float4 *>(p) = make_float4(in[0], in[1], in[2], in[3]);
    }
    __device__ __forceinline__ static uint4 pack(const float in[4])
    {
        return make_uint4(__float_as_uint(in[0]), __float_as_uint(in[1]), __float_as_uint(in[2]),
                          __float_as_uint(in[3]));
    }
    __device__ __forceinline__ static void unpack(const uint4 a, float out[4])
    {
        out[0] = __uint_as_float(a.x); out[1] = __uint_as_float(a.y);
        out[2] = __uint_as_float(a.z); out[3] = __uint_as_float(a.w);
    }
    // y[e] += element e of a raw 16-byte vector
    __device__ __forceinline__ static void add_to(const uint4 a, float y[4])
    {
        y[0] += __uint_as_float(a.x); y[1] += __uint_as_float(a.y);
        y[2] += __uint_as_float(a.z); y[3] += __uint_as_float(a.w);
    }
    // streaming (evict-first) variants for data touched once per step
    __device__ __forceinline__ static void load_cs(const float *p, float out[4])
    {
        const float4 a = __ldcs(reinterpret_cast<const float4 *>(p));
        out[0] = a.x; out[1] = a.y; out[2] = a.z; out[3] = a.w;
    }
    __device__ __forceinline__ static void store_cs(float *p, const float in[4])
    {
        __stcs(reinterpret_cast<float4 *>(p), make_float4(in[0], in[1], in[2], in[3]));
    }
};

template <>
struct VecT<__nv_bfloat16> {
    static constexpr int N = 8;
    __device__ __forceinline__ static void unpack(const uint4 a, float out[8])
    {
        const uint32_t u[4] = {a.x, a.y, a.z, a.w};
#pragma unroll
        for (int k = 0; k < 4; ++k) {
            out[2 * k] = __uint_as_float(u[k] << 16);
            out[2 * k + 1] = __uint_as_float(u[k] & 0xFFFF0000u);
        }
    }
    // y[e] += element e of a raw 16-byte vector, with the mixed-precision add
    // (the BF16 operand widens exactly, so this equals unpack-then-add)
    __device__ __forceinline__ static void add_to(const uint4 a, float y[8])
    {
        const uint32_t u[4] = {a.x, a.y, a.z, a.w};
#pragma unroll
        for (int k = 0; k < 4; ++k)
            asm("{\n\t.reg .b16 lo, hi;\n\tmov.b32 {lo, hi}, %2;\n\t"
                "add.rn.f32.bf16 %0, lo, %0;\n\tadd.rn.f32.bf16 %1, hi, %1;\n\t}"
                : "+f"(y[2 * k]), "+f"(y[2 * k + 1])
                : "r"(u[k]));
    }
    __device__ __forceinline__ static void load(const __nv_bfloat16 *p, float out[8])
    {
        unpack(*reinterpret_cast<const uint4 *>(p), out);
    }
    __device__ __forceinline__ static void load_ro(const __nv_bfloat16 *p, float out[8])
    {
        unpack(__ldg(reinterpret_cast<const uint4 *>(p)), out);
    }
    __device__ __forceinline__ static uint4 pack(const float in[8])
    {
        uint32_t u[4];
#pragma unroll
        for (int k = 0; k < 4; ++k) {
            const __nv_bfloat162 h = __floats2bfloat162_rn(in[2 * k], in[2 * k + 1]);
            u[k] = *reinterpret_cast<const uint32_t *>(&h);
        }
        return make_uint4(u[0], u[1], u[2], u[3]);
    }
    __device__ __forceinline__ static void store(__nv_bfloat16 *p, const float in[8])
    {
        *reinterpret_cast<uint4 *>(p) = pack(in);
    }
    __device__ __forceinline__ static void load_cs(const __nv_bfloat16 *p, float out[8])
    {
        unpack(__ldcs(reinterpret_cast<const uint4 *>(p)), out);
    }
    __device__ __forceinline__ static void store_cs(__nv_bfloat16 *p, const float in[8])
    {
        __stcs(reinterpret_cast<uint4 *>(p), pack(in));
    }
};

// ---------------------------------------------------------------------------
// Host-side launch entry points implemented in the .cu files.
// ---------------------------------------------------------------------------
struct StepLaunch {
    const InstDesc *descs;
    const Tile *tiles;
    const int32_t *num_tiles;
    RunStatus *status;
    int32_t r;              // offset of this launch inside its chunk (t = desc.t + r)
    int32_t grid, block;
    int32_t group_lanes, vec_per_lane;
    cudaStream_t stream;
};

// Returns false if no kernel exists for (prec, group_lanes, vec_per_lane).
bool launch_step(int32_t prec, const StepLaunch &L);
bool step_variant_exists(int32_t prec, int32_t group_lanes, int32_t vec_per_lane);
int step_max_active_blocks(int32_t prec, int32_t group_lanes, int32_t vec_per_lane, int32_t block);

void launch_init(const InstDesc *descs, int32_t slot, int32_t n, int32_t S_pad, int32_t prec, cudaStream_t st);
// dense tensor-core path: adjacency from CSR, state planes from X[t & 1]
void launch_dense_adjacency(const InstDesc *descs, int32_t slot, int32_t n, cudaStream_t st);
void launch_dense_planes(const InstDesc *descs, int32_t slot, int32_t n, int32_t S_pad, cudaStream_t st);
// max-clique column sums (fixed summation order): slots = device list of
// `count` slots (or nullptr: the one slot `slot0`); after = 1 sums the state
// written by step d.t + r, after = 0 the current state p^{d.t}
void launch_colsum(const InstDesc *descs, const int32_t *slots, int32_t count, int32_t slot0, int32_t S_max_pad,
                   int32_t prec, int32_t r, int32_t after, cudaStream_t st);
void launch_advance(InstDesc *descs, int32_t capacity, int32_t nsteps, cudaStream_t st);
void launch_prepare(const InstDesc *descs, int32_t capacity, int32_t nsteps, cudaStream_t st);
// rounding, exact costs, best replica: n_max the largest active n, total_rows the sum of active n
// dense: the run keeps the tensor-core step's adjacency bitsets (costs by popcount)
void launch_eval(const InstDesc *descs, int32_t capacity, int32_t n_max, int64_t total_rows, int32_t S_max_pad,
                 int32_t prec, bool dense, int32_t seg_max, cudaStream_t st);
void launch_pack_state(const InstDesc *descs, int32_t slot, int32_t n, int32_t S, int32_t S_pad, int32_t prec,
                       int32_t which, float *dst, cudaStream_t st);
void launch_unpack_state(const InstDesc *descs, int32_t slot, int32_t n, int32_t S, int32_t S_pad, int32_t prec,
                         const float *X, const float *m, const float *v, int32_t t, cudaStream_t st);
void launch_copy_grad(const InstDesc *descs, int32_t slot, int32_t n, int32_t S, int32_t S_pad, const float *src,
                      float *dst, cudaStream_t st);

}  // namespace qqa
