// api.cu -- host side of libqqa: the C ABI declared in include/qqa.h.
//
// A qqa_problem is a validated device copy of one CSR graph. A qqa_run is a
// table of instance slots (one InstDesc per slot in device memory), the list
// of (slot, row-block) tiles the fused step kernel walks, and the CUDA graphs
// that replay chunks of steps. Every step of the method runs in the kernels of
// step_*.cu and aux_kernels.cu; this file validates arguments, allocates,
// builds descriptors and tiles, and launches.
#include <algorithm>
#include <cmath>
#include <cstdarg>
#include <cstdio>
#include <cstring>
#include <map>
#include <mutex>
#include <new>
#include <string>
#include <atomic>
#include <vector>

#include <cuda.h>
#include <cudaTypedefs.h>

#include "../../include/qqa.h"
#include "qqa_internal.cuh"

namespace qqa {
using StepFn = void (*)(const InstDesc *, const Tile *, const int32_t *, RunStatus *, int32_t);
using TiledFn = void (*)(const InstDesc *, const Tile *, const int32_t *, RunStatus *, int32_t, int32_t, int32_t);
StepFn step_kernel_fp32(int G, int VPL);
StepFn step_kernel_bf16(int G, int VPL);
TiledFn step_tiled_kernel_fp32(int G, int VPL, int RPW);
TiledFn step_tiled_kernel_bf16(int G, int VPL, int RPW);
StepFn step_stream_kernel_fp32(int G, int VPL, int NB);
StepFn step_stream_kernel_bf16(int G, int VPL, int NB);
StepFn dense_gemm_kernel(int N);
using UpdFn = void (*)(const InstDesc *, const Tile *, const int32_t *, RunStatus *, int32_t, int32_t);
UpdFn dense_update_kernel(int prec, int G, int VPL);
using PipeFn = void (*)(const InstDesc *, const Tile *, const int32_t *, RunStatus *, int32_t, int32_t);
PipeFn step_pipe_kernel_fp32(int G, int VPL, bool segs);
PipeFn step_pipe_kernel_bf16(int G, int VPL, bool segs);
StepFn step_hub_kernel_fp32(int G, int VPL);
StepFn step_hub_kernel_bf16(int G, int VPL);
StepFn step_scalar_kernel(int prec, int L);
int dense_gemm_threads();
int dense_smem_bytes(int N);
}  // namespace qqa

using namespace qqa;

// ------------------------------------------------------------------ errors
static thread_local std::string g_last_error;
static std::atomic<unsigned long long> g_launches{0};

static int fail(int code, const char *fmt, ...)
{
    char buf[1024];
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(buf, sizeof buf, fmt, ap);
    va_end(ap);
    g_last_error = buf;
    return code;
}

#define QQA_CK(call)                                                                          \
    do {                                                                                      \
        cudaError_t e_ = (call);                                                              \
        if (e_ != cudaSuccess) return fail(QQA_ECUDA, "%s: %s", #call, cudaGetErrorString(e_)); \
    } while (0)

#define QQA_CK_LAUNCH(what)                                                                   \
    do {                                                                                      \
        cudaError_t e_ = cudaGetLastError();                                                  \
        if (e_ != cudaSuccess) return fail(QQA_ECUDA, "%s launch: %s", what, cudaGetErrorString(e_)); \
    } while (0)

// --------------------------------------------------------------- allocator
struct Alloc {
    qqa_allocator user{};
    bool has_user = false;
    void *get(size_t bytes, cudaStream_t st)
    {
        if (bytes == 0) bytes = 16;
        if (has_user) return user.alloc(bytes, (void *)st, user.ctx);
        void *p = nullptr;
        if (cudaMalloc(&p, bytes) != cudaSuccess) {
            (void)cudaGetLastError();
            return nullptr;
        }
        return p;
    }
    void put(void *p, cudaStream_t st)
    {
        if (!p) return;
        if (has_user) user.free(p, (void *)st, user.ctx);
        else cudaFree(p);
    }
    static Alloc from(const qqa_allocator *a)
    {
        Alloc r;
        if (a && a->alloc && a->free) {
            r.user = *a;
            r.has_user = true;
        }
        return r;
    }
};

struct qqa_problem {
    int32_t kind = 0, n = 0;
    int64_t nnz = 0;
    int32_t max_abs_w = 1;   // largest |edge weight| (1 when unweighted)
    int32_t *row_ptr = nullptr, *col = nullptr, *w = nullptr;
    // long rows: degree above long_thresh, summed in segments of kSegLen
    // neighbours by the long-row kernel (device tables; none when nlong = 0)
    int32_t long_thresh = 0x7fffffff, nlong = 0, nseg = 0;
    int32_t *long_rows = nullptr, *seg_ptr = nullptr, *seg_row = nullptr;
    // graphs with a wide spread of degrees (the largest row below the long-row
    // threshold at least 4x the mean): each row's degree, 0 for long rows (host
    // copy; empty otherwise). The pipelined kernel's tile list is ordered by it.
    std::vector<uint16_t> short_deg;
    Alloc alloc;
};

// A row is long when its degree exceeds max(64, 8 x the mean degree rounded
// up): on graphs with hubs (scale-free degree distributions) such a row would
// take a lane group many times longer than a typical row.
static int32_t long_row_threshold(int32_t n, int64_t nnz)
{
    const int64_t mean_up = (nnz + n - 1) / std::max<int32_t>(n, 1);
    return (int32_t)std::min<int64_t>(0x7fffffff, std::max<int64_t>(64, 8 * mean_up));
}

// ------------------------------------------------------------------- misc
extern "C" const char *qqa_last_error(void) { return g_last_error.c_str(); }
extern "C" const char *qqa_version(void) { return "qqa-gb300 0.1 (sm_103a)"; }
extern "C" uint64_t qqa_launch_count(void) { return g_launches.load(); }

extern "C" void qqa_default_params(qqa_params *p)
{
    if (!p) return;
    std::memset(p, 0, sizeof *p);
    p->S = 128;
    p->steps = 3000;
    p->round_every = 50;
    p->a_ent = 4;
    p->lr = 0.1f;
    p->weight_decay = 0.01f;
    p->beta1 = 0.9f;
    p->beta2 = 0.999f;
    p->adam_eps = 1e-8f;
    p->gamma_min = -2.0f;
    p->gamma_max = 0.1f;
    p->alpha_comm = 0.1f;
    p->comm_eps = 1e-8f;
    p->temperature = 1e-3f;
    p->lambda = 2.0f;
    p->seed = 0;
    p->precision = QQA_FP32;
}

extern "C" int qqa_device_sm_count(void)
{
    int dev = 0, sms = 0;
    QQA_CK(cudaGetDevice(&dev));
    QQA_CK(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));
    return sms;
}

// --------------------------------------------------------------- problems
static int validate_csr(int32_t kind, int32_t n, const int32_t *rp, const int32_t *col, const int32_t *w)
{
    if (kind < QQA_MIS || kind > QQA_MAXCLIQUE) return fail(QQA_EINVAL, "unknown problem kind %d", kind);
    if (n < 1) return fail(QQA_EINVAL, "n must be >= 1 (got %d)", n);
    if (!rp) return fail(QQA_EINVAL, "row_ptr is NULL");
    if (rp[0] != 0) return fail(QQA_EINVAL, "row_ptr[0] must be 0");
    for (int32_t i = 0; i < n; ++i)
        if (rp[i + 1] < rp[i]) return fail(QQA_EINVAL, "row_ptr decreases at row %d", i);
    const int64_t nnz = rp[n];
    if (nnz > 0 && !col) return fail(QQA_EINVAL, "col is NULL");
    if (w && kind != QQA_MAXCUT) return fail(QQA_EINVAL, "edge weights are only defined for max-cut");
    for (int32_t i = 0; i < n; ++i) {
        for (int64_t k = rp[i]; k < rp[i + 1]; ++k) {
            const int32_t j = col[k];
            if (j < 0 || j >= n) return fail(QQA_EINVAL, "col[%lld] = %d out of range [0, %d)", (long long)k, j, n);
            if (j == i) return fail(QQA_EINVAL, "self-loop at node %d", i);
            if (k > rp[i] && col[k - 1] >= j) return fail(QQA_EINVAL, "row %d not strictly increasing", i);
        }
    }
    // Symmetry in O(nnz): scatter every entry (i, j) into row j of the
    // transpose; visiting i in increasing order leaves each transposed row
    // sorted, so the graph is symmetric exactly when the transpose equals it
    // (and the weights of (i, j) and (j, i) agree). Only when it does not is
    // the offending entry looked for (by binary search), for the message.
    auto report_asymmetry = [&]() -> int {
        for (int32_t i = 0; i < n; ++i)
            for (int64_t k = rp[i]; k < rp[i + 1]; ++k) {
                const int32_t j = col[k];
                const int32_t *b = col + rp[j], *e = col + rp[j + 1];
                const int32_t *f = std::lower_bound(b, e, i);
                if (f == e || *f != i) return fail(QQA_EINVAL, "edge (%d,%d) has no reverse entry", i, j);
                if (w && w[k] != w[f - col])
                    return fail(QQA_EINVAL, "weight of (%d,%d) differs from (%d,%d)", i, j, j, i);
            }
        return fail(QQA_EINVAL, "the graph is not symmetric");
    };
    std::vector<int64_t> pos(rp, rp + n);
    for (int64_t k = 0; k < nnz; ++k) ++pos[col[k]];   // row starts + in-degrees
    for (int32_t j = 0; j < n; ++j)
        if (pos[j] != rp[j + 1]) return report_asymmetry();   // in-degree != out-degree
    std::copy(rp, rp + n, pos.begin());
    std::vector<int32_t> tcol((size_t)nnz), tw(w ? (size_t)nnz : 0);
    for (int32_t i = 0; i < n; ++i)
        for (int64_t k = rp[i]; k < rp[i + 1]; ++k) {
            const int64_t p = pos[col[k]]++;
            tcol[p] = i;
            if (w) tw[p] = w[k];
        }
    for (int64_t k = 0; k < nnz; ++k)
        if (tcol[k] != col[k] || (w && tw[k] != w[k])) return report_asymmetry();
    return QQA_OK;
}

// Shared with the colouring entry points (color.cu): the error slot, the
// graph checks (unit weights) and the launch counter of this library.
namespace qqa {
int set_error(int code, const char *msg) { return fail(code, "%s", msg); }
int check_unit_graph(int32_t n, const int32_t *rp, const int32_t *col) { return validate_csr(QQA_MIS, n, rp, col, nullptr); }
void add_launches(unsigned long long k) { g_launches += k; }
}  // namespace qqa

extern "C" int qqa_create_problem(int32_t kind, int32_t n, const int32_t *row_ptr, const int32_t *col,
                                  const int32_t *w, const qqa_allocator *alloc, void *stream, qqa_problem **out)
{
    if (!out) return fail(QQA_EINVAL, "out is NULL");
    *out = nullptr;
    int rc = validate_csr(kind, n, row_ptr, col, w);
    if (rc) return rc;
    cudaStream_t st = (cudaStream_t)stream;
    qqa_problem *p = new (std::nothrow) qqa_problem();
    if (!p) return fail(QQA_ENOMEM, "host allocation failed");
    p->kind = kind;
    p->n = n;
    p->nnz = row_ptr[n];
    if (w)
        for (int64_t k = 0; k < p->nnz; ++k) p->max_abs_w = std::max(p->max_abs_w, w[k] < 0 ? -w[k] : w[k]);
    p->alloc = Alloc::from(alloc);
    // long rows and their segments
    std::vector<int32_t> lrows, lseg_ptr{0}, lseg_row;
    p->long_thresh = long_row_threshold(n, p->nnz);
    for (int32_t i = 0; i < n; ++i) {
        const int32_t deg = row_ptr[i + 1] - row_ptr[i];
        if (deg <= p->long_thresh) continue;
        const int32_t nsegs = (deg + kSegLen - 1) / kSegLen;
        for (int32_t q = 0; q < nsegs; ++q) lseg_row.push_back((int32_t)lrows.size());
        lrows.push_back(i);
        lseg_ptr.push_back(lseg_ptr.back() + nsegs);
    }
    p->nlong = (int32_t)lrows.size();
    p->nseg = (int32_t)lseg_row.size();
    {
        int32_t max_short = 0;
        for (int32_t i = 0; i < n; ++i) {
            const int32_t deg = row_ptr[i + 1] - row_ptr[i];
            if (deg <= p->long_thresh) max_short = std::max(max_short, deg);
        }
        const int64_t mean_up = (p->nnz + n - 1) / std::max<int32_t>(n, 1);
        if (n > 0 && (int64_t)max_short >= 4 * std::max<int64_t>(mean_up, 1)) {
            p->short_deg.resize((size_t)n);
            for (int32_t i = 0; i < n; ++i) {
                const int32_t deg = row_ptr[i + 1] - row_ptr[i];
                p->short_deg[(size_t)i] = deg > p->long_thresh ? 0 : (uint16_t)std::min(deg, 65535);
            }
        }
    }
    p->row_ptr = (int32_t *)p->alloc.get(sizeof(int32_t) * (size_t)(n + 1), st);
    p->col = (int32_t *)p->alloc.get(sizeof(int32_t) * (size_t)std::max<int64_t>(p->nnz, 1), st);
    if (w) p->w = (int32_t *)p->alloc.get(sizeof(int32_t) * (size_t)std::max<int64_t>(p->nnz, 1), st);
    if (p->nlong) {
        p->long_rows = (int32_t *)p->alloc.get(sizeof(int32_t) * (size_t)p->nlong, st);
        p->seg_ptr = (int32_t *)p->alloc.get(sizeof(int32_t) * (size_t)(p->nlong + 1), st);
        p->seg_row = (int32_t *)p->alloc.get(sizeof(int32_t) * (size_t)p->nseg, st);
    }
    if (!p->row_ptr || !p->col || (w && !p->w) || (p->nlong && (!p->long_rows || !p->seg_ptr || !p->seg_row))) {
        qqa_destroy_problem(p);
        return fail(QQA_ENOMEM, "device allocation for the graph failed");
    }
    cudaError_t e = cudaMemcpyAsync(p->row_ptr, row_ptr, sizeof(int32_t) * (size_t)(n + 1), cudaMemcpyHostToDevice, st);
    if (e == cudaSuccess && p->nnz)
        e = cudaMemcpyAsync(p->col, col, sizeof(int32_t) * (size_t)p->nnz, cudaMemcpyHostToDevice, st);
    if (e == cudaSuccess && w && p->nnz)
        e = cudaMemcpyAsync(p->w, w, sizeof(int32_t) * (size_t)p->nnz, cudaMemcpyHostToDevice, st);
    if (e == cudaSuccess && p->nlong)
        e = cudaMemcpyAsync(p->long_rows, lrows.data(), sizeof(int32_t) * lrows.size(), cudaMemcpyHostToDevice, st);
    if (e == cudaSuccess && p->nlong)
        e = cudaMemcpyAsync(p->seg_ptr, lseg_ptr.data(), sizeof(int32_t) * lseg_ptr.size(), cudaMemcpyHostToDevice, st);
    if (e == cudaSuccess && p->nlong)
        e = cudaMemcpyAsync(p->seg_row, lseg_row.data(), sizeof(int32_t) * lseg_row.size(), cudaMemcpyHostToDevice, st);
    if (e == cudaSuccess) e = cudaStreamSynchronize(st);  // host arrays may be freed after return
    if (e != cudaSuccess) {
        qqa_destroy_problem(p);
        return fail(QQA_ECUDA, "graph upload: %s", cudaGetErrorString(e));
    }
    *out = p;
    return QQA_OK;
}

extern "C" int qqa_problem_info(const qqa_problem *p, int32_t *kind, int32_t *n, int64_t *nnz)
{
    if (!p) return fail(QQA_EINVAL, "problem is NULL");
    if (kind) *kind = p->kind;
    if (n) *n = p->n;
    if (nnz) *nnz = p->nnz;
    return QQA_OK;
}

extern "C" void qqa_destroy_problem(qqa_problem *p)
{
    if (!p) return;
    p->alloc.put(p->row_ptr, 0);
    p->alloc.put(p->col, 0);
    p->alloc.put(p->w, 0);
    p->alloc.put(p->long_rows, 0);
    p->alloc.put(p->seg_ptr, 0);
    p->alloc.put(p->seg_row, 0);
    delete p;
}

// -------------------------------------------------------------------- runs
struct SlotHost {
    bool active = false;
    const qqa_problem *prob = nullptr;
    qqa_params prm{};
    int32_t n = 0, S = 0, S_pad = 0, W = 0, K = 0;
    int32_t t = 0;            // exact host mirror of the device step counter
    int32_t last_eval_t = -1; // host mirror of the evaluation rule
    int32_t hist_cap = 0;
    std::vector<void *> dev;  // device allocations of this slot
    // host mirrors of the latest evaluation (filled by qqa_run_sync)
    std::vector<long long> obj, viol;
    std::vector<uint8_t> feas;
    std::vector<double> energy;
    int32_t best = -1, eval_step = -1, eval_count = 0;
};

// chains of a tensor-core run (see qqa_run::nchains): at most kMaxChains, kChains used
static constexpr int kMaxChains = 4;
static constexpr int kChains = 4;

struct qqa_run {
    int32_t capacity = 0, S_max = 0, S_max_pad = 0, prec = 0, vec = 4;
    qqa_launch_config cfg{};
    int32_t rows_per_tile = 0, max_grid = 0, smem = 0;
    StepFn step_fn = nullptr;
    bool scalar = false;              // one replica per instance: state p[n], scalar kernel
    int32_t mean_deg_hint = 0;        // mean degree of the instances (scalar kernel's lanes per row)
    StepFn hub_fn = nullptr;          // long-row kernel for the (G, VPL) of the step kernel
    int32_t hub_max_grid = 0;
    Tile *d_hub_items = nullptr;      // (slot, segment) work items of the long-row kernel
    int32_t hub_cap = 0, num_hub_items = 0, hub_grid = 0;
    int32_t *d_clique_slots = nullptr;   // active max-clique slots (column sums after every step)
    int32_t clique_cap = 0, num_clique = 0;
    int32_t kernels_per_step = 1;
    bool dynamic = false;             // slots come and go: always launch the full persistent grid
    int32_t dense_N = 0;              // > 0: tensor-core step (MMA width = replicas covered)
    UpdFn upd_fn = nullptr;           // its update kernel (32-row tiles of the second list)
    int32_t upd_block = 256, upd_max_grid = 0, upd_smem = 0, upd_ld = 0;
    Tile *d_tiles2 = nullptr;         // the update kernel's tiles
    int32_t tile2_cap = 0, num_tiles2 = 0;
    TiledFn tiled_fn = nullptr;       // set when the TMA-staged kernel is used
    PipeFn pipe_fn = nullptr;         // set when the pipelined kernel is used
    PipeFn pipe_seg_fn = nullptr;     // its variant that also takes segment work items of long rows
    bool seg_items = false;           // the tile list holds segment work items (pipe_seg_fn runs)
    int32_t pipe_buf = 0;             // bytes of one of its two shared-memory buffers
    int32_t chunk_rows = 0, buf_elems = 0;
    Alloc alloc;
    InstDesc *d_descs = nullptr;
    std::vector<InstDesc> h_descs;
    Tile *d_tiles = nullptr;
    int32_t tile_cap = 0;
    int32_t *d_num_tiles = nullptr;  // [0] tiles, [1] streaming cache hints on (state larger than L2), [2] long-row items,
                                     // [3] update tiles; chained tensor-core runs: [4 + c] product tiles of chain c,
                                     // [4 + kMaxChains + c] its update tiles
    int32_t tile_words[4 + 2 * kMaxChains] = {};
    // Tensor-core runs of several instances: the instances form up to
    // kMaxChains chains of about equal row tiles, each launched on its own
    // stream (forked from the caller's and joined back after the chunk). A
    // chain's step waits only for its own previous step, so one chain's update
    // runs beside another's product (the product kernel fills few SMs and
    // waits on its loads) instead of after the product of every instance.
    int32_t nchains = 1;
    int32_t chain_t0[kMaxChains + 1] = {}, chain_u0[kMaxChains + 1] = {};   // first product / update tile of each chain
    cudaStream_t chain_st[kMaxChains] = {};   // chains 1.. (chain 0 runs on the caller's stream)
    cudaEvent_t ev_fork = nullptr, ev_join[kMaxChains] = {};
    int32_t num_tiles = 0;
    RunStatus *d_status = nullptr;
    float *d_scratch = nullptr;   // state import/export staging
    size_t scratch_bytes = 0;
    std::vector<SlotHost> slots;
    cudaStream_t cap_stream = nullptr;
    std::map<std::pair<int, int>, cudaGraphExec_t> graphs;
};

static const bool kAutoStaged = false;
static const int kTiledIdxCapHost = 8192;   // must equal kTiledIdxCap in step_impl.cuh

static int pick_layout(int32_t S_pad, int32_t vec, int32_t &G, int32_t &VPL)
{
    const int nvec = S_pad / vec;
    if (nvec <= 32) {
        G = 1;
        while (G < nvec) G <<= 1;
        VPL = 1;
    } else {
        G = 32;
        VPL = 1;
        while (G * VPL < nvec) VPL <<= 1;
    }
    return QQA_OK;
}

// staged_hint: 1 if the graphs favour the staged kernel (auto mode), else 0.
static int resolve_scalar(qqa_run *r, qqa_launch_config c)
{
    if (c.kernel != QQA_KERNEL_AUTO && c.kernel != QQA_KERNEL_SCALAR)
        return fail(QQA_EINVAL, "runs of one replica per instance use the scalar kernel (QQA_KERNEL_SCALAR)");
    int L = c.kernel_param;
    if (L == 0) {
        const int md = r->mean_deg_hint;
        L = md <= 6 ? 4 : (md <= 24 ? 8 : (md <= 64 ? 16 : 32));
    }
    r->step_fn = step_scalar_kernel(r->prec, L);
    if (!r->step_fn) return fail(QQA_EINVAL, "no scalar kernel with %d lanes per row (4, 8, 16, 32)", L);
    const int block = c.block_threads ? c.block_threads : 256;
    if (block < 32 || block > 256 || block % 32)
        return fail(QQA_EINVAL, "block_threads must be a multiple of 32 in [32, 256]");
    int dev = 0, sms = 0, occ = 0;
    QQA_CK(cudaGetDevice(&dev));
    QQA_CK(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));
    QQA_CK(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, r->step_fn, block, 0));
    if (occ < 1) return fail(QQA_EINVAL, "scalar kernel cannot run %d threads per block", block);
    r->scalar = true;
    r->tiled_fn = nullptr;
    r->pipe_fn = nullptr;
    r->pipe_seg_fn = nullptr;
    r->hub_fn = nullptr;
    r->upd_fn = nullptr;
    r->dense_N = 0;
    r->smem = 0;
    r->rows_per_tile = block;   // 32 rows per warp
    c.group_lanes = L;
    c.vec_per_lane = 1;
    c.block_threads = block;
    c.kernel = QQA_KERNEL_SCALAR;
    c.kernel_param = L;
    r->max_grid = c.grid_blocks ? c.grid_blocks : sms * occ;
    c.grid_blocks = r->max_grid;
    r->cfg = c;
    return QQA_OK;
}

// The long-row kernel of the step kernel's (G, VPL), for runs that gather
// neighbour rows (not the tensor-core or scalar steps).
static int resolve_hub(qqa_run *r, int32_t G, int32_t VPL)
{
    r->hub_fn = r->prec == kFP32 ? step_hub_kernel_fp32(G, VPL) : step_hub_kernel_bf16(G, VPL);
    if (!r->hub_fn) return fail(QQA_EINVAL, "no long-row kernel for G=%d VPL=%d", G, VPL);
    int dev = 0, sms = 0, occ = 0;
    QQA_CK(cudaGetDevice(&dev));
    QQA_CK(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));
    QQA_CK(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, r->hub_fn, 256, 0));
    if (occ < 1) return fail(QQA_EINVAL, "long-row kernel G=%d VPL=%d does not fit on an SM", G, VPL);
    r->hub_max_grid = sms * occ;
    return QQA_OK;
}

static int resolve_config(qqa_run *r, const qqa_launch_config *cfg, int staged_hint)
{
    qqa_launch_config c{};
    if (cfg) c = *cfg;
    if (r->S_max == 1) return resolve_scalar(r, c);
    int32_t G = c.group_lanes, VPL = c.vec_per_lane;
    if (G == 0 || VPL == 0) {
        int32_t g2, v2;
        pick_layout(r->S_max_pad, r->vec, g2, v2);
        if (G == 0 && VPL == 0) { G = g2; VPL = v2; }
        else if (G == 0) { G = 1; while (G < 32 && G * VPL * r->vec < r->S_max_pad) G <<= 1; }
        else { VPL = 1; while (G * VPL * r->vec < r->S_max_pad) VPL <<= 1; }
    }
    if (G * VPL * r->vec < r->S_max_pad)
        return fail(QQA_EINVAL, "layout G=%d VPL=%d covers %d replicas < %d", G, VPL, G * VPL * r->vec, r->S_max_pad);
    int mode = c.kernel;
    if (mode == QQA_KERNEL_AUTO)
        mode = (staged_hint && (c.block_threads == 0 || c.block_threads == 256)) ? QQA_KERNEL_STAGED : QQA_KERNEL_DIRECT;
    if (mode == QQA_KERNEL_AUTO) mode = QQA_KERNEL_DIRECT;
    if (mode < QQA_KERNEL_DIRECT || mode > QQA_KERNEL_PIPE) return fail(QQA_EINVAL, "unknown kernel %d", c.kernel);
    r->pipe_fn = nullptr;
    r->pipe_seg_fn = nullptr;
    r->hub_fn = nullptr;
    if (mode == QQA_KERNEL_DENSE) {
        const int N = r->S_max_pad <= 64 ? 64 : (r->S_max_pad <= 128 ? 128 : (r->S_max_pad <= 256 ? 256 : 0));
        if (!N) return fail(QQA_EINVAL, "the dense tensor-core step covers at most 256 replicas");
        r->step_fn = dense_gemm_kernel(N);
        r->tiled_fn = nullptr;
        r->dense_N = N;
        r->smem = dense_smem_bytes(N);
        const int block_d = dense_gemm_threads();
        int dev = 0, sms = 0, occ = 0, occ_u = 0;
        QQA_CK(cudaGetDevice(&dev));
        QQA_CK(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));
        QQA_CK(cudaFuncSetAttribute(r->step_fn, cudaFuncAttributeMaxDynamicSharedMemorySize, r->smem));
        QQA_CK(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, r->step_fn, block_d, r->smem));
        if (occ < 1) return fail(QQA_EINVAL, "dense step kernel does not fit on an SM");
        // the update kernel: up to 16 replicas per lane (the epilogue's
        // per-row work is shared by more elements), as many lanes as cover S
        int32_t Vu = 16 / r->vec;   // 4 FP32 or 2 BF16 vectors
        int32_t nvec = 1;
        while (nvec * r->vec < r->S_max_pad) nvec <<= 1;
        Vu = std::min(Vu, nvec);
        const int32_t Gu = nvec / Vu;
        r->upd_fn = dense_update_kernel(r->prec, Gu, Vu);
        if (!r->upd_fn) return fail(QQA_EINVAL, "no tensor-core update kernel for G=%d VPL=%d", Gu, Vu);
        r->upd_ld = r->S_max_pad + 1;   // odd row stride of the shared buffer: conflict-free transposition
        r->upd_smem = 32 * r->upd_ld * (int)sizeof(float);
        QQA_CK(cudaFuncSetAttribute(r->upd_fn, cudaFuncAttributeMaxDynamicSharedMemorySize, r->upd_smem));
        QQA_CK(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ_u, r->upd_fn, r->upd_block, r->upd_smem));
        if (occ_u < 1) return fail(QQA_EINVAL, "dense update kernel does not fit on an SM");
        r->upd_max_grid = sms * occ_u;
        r->rows_per_tile = 128;
        c.group_lanes = Gu;
        c.vec_per_lane = Vu;
        c.block_threads = block_d;
        c.kernel = mode;
        c.kernel_param = N;
        r->max_grid = c.grid_blocks ? c.grid_blocks : sms * occ;
        c.grid_blocks = r->max_grid;
        r->cfg = c;
        return QQA_OK;
    }
    int rpw = c.kernel_param ? c.kernel_param : (mode == QQA_KERNEL_STREAM ? 8 : 4);
    if (mode == QQA_KERNEL_STAGED) {
        r->tiled_fn = r->prec == kFP32 ? step_tiled_kernel_fp32(G, VPL, rpw) : step_tiled_kernel_bf16(G, VPL, rpw);
        if (!r->tiled_fn) {
            if (c.kernel == QQA_KERNEL_STAGED)
                return fail(QQA_EINVAL, "no staged kernel for G=%d VPL=%d rows_per_warp=%d", G, VPL, rpw);
            mode = QQA_KERNEL_DIRECT;   // auto: fall back to the direct-gather kernel
        }
    }
    const int tb = r->prec == kFP32 ? 4 : 2;
    int block = c.block_threads ? c.block_threads : 256;
    int dev = 0, sms = 0, occ = 0;
    QQA_CK(cudaGetDevice(&dev));
    QQA_CK(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));
    if (mode == QQA_KERNEL_STAGED) {
        if (c.block_threads && c.block_threads != 256) return fail(QQA_EINVAL, "the staged kernel runs 256 threads");
        block = 256;
        const int row_bytes = r->S_max_pad * tb;
        r->chunk_rows = std::max(8, 32768 / row_bytes);
        r->buf_elems = r->chunk_rows * r->S_max_pad;
        // header, two chunk buffers, CSR index segment
        r->smem = 128 + 2 * r->buf_elems * tb + kTiledIdxCapHost * (int)sizeof(int32_t);
        QQA_CK(cudaFuncSetAttribute(r->tiled_fn, cudaFuncAttributeMaxDynamicSharedMemorySize, r->smem));
        QQA_CK(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, r->tiled_fn, block, r->smem));
        r->rows_per_tile = (block / 32) * rpw * (32 / G);
        r->step_fn = nullptr;
    } else if (mode == QQA_KERNEL_PIPE) {
        r->tiled_fn = nullptr;
        r->step_fn = nullptr;
        rpw = 0;
        r->pipe_fn = r->prec == kFP32 ? step_pipe_kernel_fp32(G, VPL, false) : step_pipe_kernel_bf16(G, VPL, false);
        r->pipe_seg_fn = r->prec == kFP32 ? step_pipe_kernel_fp32(G, VPL, true) : step_pipe_kernel_bf16(G, VPL, true);
        if (!r->pipe_fn || !r->pipe_seg_fn) return fail(QQA_EINVAL, "no pipelined kernel for G=%d VPL=%d", G, VPL);
        if (block < 32 || block > 256 || block % 32)
            return fail(QQA_EINVAL, "block_threads must be a multiple of 32 in [32, 256]");
        // every warp owns two buffers, each holding one tile's rows of p (FP32),
        // m and v; a tile is the warp's 32 / G rows (one per lane group)
        auto smem_for = [&](int b, int32_t &buf) {
            buf = (32 / G) * r->S_max_pad * (4 + 2 * tb);
            return 128 + (b / 32) * 2 * buf;
        };
        int max_smem = 0;
        QQA_CK(cudaDeviceGetAttribute(&max_smem, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev));
        if (c.block_threads == 0) {
            int best_warps = -1;
            for (int b : {256, 128, 64}) {
                int32_t buf = 0;
                const int sm = smem_for(b, buf);
                if (sm > max_smem) continue;
                int o = 0;
                QQA_CK(cudaFuncSetAttribute(r->pipe_fn, cudaFuncAttributeMaxDynamicSharedMemorySize, sm));
                QQA_CK(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&o, r->pipe_fn, b, sm));
                if (o * b / 32 > best_warps) { best_warps = o * b / 32; block = b; }
            }
        }
        r->smem = smem_for(block, r->pipe_buf);
        if (r->smem > max_smem)
            return fail(QQA_EINVAL, "pipelined kernel needs %d bytes of shared memory (S=%d, %d threads)", r->smem,
                        r->S_max_pad, block);
        QQA_CK(cudaFuncSetAttribute(r->pipe_fn, cudaFuncAttributeMaxDynamicSharedMemorySize, r->smem));
        QQA_CK(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, r->pipe_fn, block, r->smem));
        int occ_seg = 0;   // the grid must be resident for either variant
        QQA_CK(cudaFuncSetAttribute(r->pipe_seg_fn, cudaFuncAttributeMaxDynamicSharedMemorySize, r->smem));
        QQA_CK(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ_seg, r->pipe_seg_fn, block, r->smem));
        occ = std::min(occ, occ_seg);
        r->rows_per_tile = 32 / G;
    } else if (mode == QQA_KERNEL_STREAM) {
        r->tiled_fn = nullptr;
        r->step_fn = r->prec == kFP32 ? step_stream_kernel_fp32(G, VPL, rpw) : step_stream_kernel_bf16(G, VPL, rpw);
        if (!r->step_fn) return fail(QQA_EINVAL, "no stream kernel for G=%d VPL=%d prefetch=%d", G, VPL, rpw);
        if (block < 32 || block > 256 || block % 32)
            return fail(QQA_EINVAL, "block_threads must be a multiple of 32 in [32, 256]");
        const int slots = (r->prec == kFP32 ? 1 : 2) + 2 + rpw;   // own p words, m, v, neighbours
        r->smem = 2 * VPL * slots * block * 16;
        QQA_CK(cudaFuncSetAttribute(r->step_fn, cudaFuncAttributeMaxDynamicSharedMemorySize, r->smem));
        QQA_CK(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, r->step_fn, block, r->smem));
        r->rows_per_tile = (block / 32) * (32 / G);
    } else {
        r->tiled_fn = nullptr;
        rpw = 0;
        r->step_fn = r->prec == kFP32 ? step_kernel_fp32(G, VPL) : step_kernel_bf16(G, VPL);
        if (!r->step_fn) return fail(QQA_EINVAL, "no step kernel for G=%d VPL=%d precision %d", G, VPL, r->prec);
        r->smem = 0;
        if (c.block_threads == 0) {
            // registers are allocated per warp: pick the block size that keeps
            // the most warps resident (ties go to the larger block)
            int best_warps = -1;
            for (int b : {256, 128, 64}) {
                int o = 0;
                QQA_CK(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&o, r->step_fn, b, r->smem));
                if (o * b / 32 > best_warps) { best_warps = o * b / 32; block = b; }
            }
        }
        if (block < 32 || block > 256 || block % 32)
            return fail(QQA_EINVAL, "block_threads must be a multiple of 32 in [32, 256]");
        QQA_CK(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, r->step_fn, block, r->smem));
        r->rows_per_tile = (block / 32) * (32 / G);
    }
    if (occ < 1) return fail(QQA_EINVAL, "step kernel G=%d VPL=%d cannot run %d threads per block", G, VPL, block);
    const int hrc = resolve_hub(r, G, VPL);
    if (hrc) return hrc;
    c.group_lanes = G;
    c.vec_per_lane = VPL;
    c.block_threads = block;
    c.kernel = mode;
    c.kernel_param = rpw;
    r->max_grid = c.grid_blocks ? c.grid_blocks : sms * occ;
    c.grid_blocks = r->max_grid;
    r->cfg = c;
    return QQA_OK;
}

static int upload_desc(qqa_run *r, int32_t slot, cudaStream_t st)
{
    // the device advances t and last_eval_t itself; the host mirrors follow the
    // same rules exactly, so re-uploading a descriptor never moves them
    r->h_descs[slot].t = r->slots[slot].t;
    r->h_descs[slot].last_eval_t = r->slots[slot].last_eval_t;
    QQA_CK(cudaMemcpyAsync(r->d_descs + slot, &r->h_descs[slot], sizeof(InstDesc), cudaMemcpyHostToDevice, st));
    QQA_CK(cudaStreamSynchronize(st));  // the host mirror may change again right after
    return QQA_OK;
}

static void drop_graphs(qqa_run *r)
{
    for (auto &kv : r->graphs) cudaGraphExecDestroy(kv.second);
    r->graphs.clear();
}

static int rebuild_tiles(qqa_run *r, cudaStream_t st)
{
    std::vector<Tile> tiles;
    // the pipelined kernel takes the segments of long rows as work items of its
    // own list, first (one segment per lane group of a warp); the other gather
    // kernels leave them to the long-row kernel
    const bool fold = r->pipe_fn != nullptr;
    if (fold)
        for (int32_t k = 0; k < r->capacity; ++k) {
            const SlotHost &s = r->slots[k];
            if (!s.active || !r->h_descs[k].hub_active) continue;
            for (int32_t q = 0; q < s.prob->nseg; q += r->rows_per_tile) tiles.push_back(Tile{k, -(q + 1)});
        }
    // Warps take the tiles round-robin, so on a graph whose row degrees spread
    // widely (scale-free) a warp's share of the gather work varies with the
    // tiles it happens to get, and the launch waits for the most loaded warp.
    // For the pipelined kernel such a slot's tiles are listed by decreasing
    // largest degree (stable, so rows of equal degree stay in order): each
    // round of the walk then takes tiles of about equal cost, and the cheapest
    // come last. The order does not change any result: rows are independent.
    std::vector<std::pair<int32_t, int32_t>> keyed;   // (key, row0)
    for (int32_t k = 0; k < r->capacity; ++k) {
        const SlotHost &s = r->slots[k];
        if (!s.active) continue;
        const std::vector<uint16_t> &sd = s.prob->short_deg;
        if (!fold || sd.empty()) {
            for (int32_t row0 = 0; row0 < s.n; row0 += r->rows_per_tile) tiles.push_back(Tile{k, row0});
            continue;
        }
        keyed.clear();
        for (int32_t row0 = 0; row0 < s.n; row0 += r->rows_per_tile) {
            int32_t key = 0;
            for (int32_t i = row0; i < std::min(s.n, row0 + r->rows_per_tile); ++i) key = std::max<int32_t>(key, sd[(size_t)i]);
            keyed.emplace_back(key, row0);
        }
        std::stable_sort(keyed.begin(), keyed.end(),
                         [](const std::pair<int32_t, int32_t> &a, const std::pair<int32_t, int32_t> &b) { return a.first > b.first; });
        for (const auto &kr : keyed) tiles.push_back(Tile{k, kr.second});
    }
    const int32_t nt = (int32_t)tiles.size();
    const bool seg_items = fold && !tiles.empty() && tiles.front().row0 < 0;
    // a list doubles when it is full and is cut to twice its entries when they
    // fall below a quarter of it, so its capacity stays within 4x its entries
    auto resize_to = [](int32_t need, int32_t cap) -> int32_t {
        if (need > cap) return std::max<int32_t>(need, 2 * cap);
        if (cap > 256 && need < cap / 4) return std::max<int32_t>(2 * need, 256);
        return cap;
    };
    if (resize_to(nt, r->tile_cap) != r->tile_cap) {
        int32_t cap = resize_to(nt, r->tile_cap);
        QQA_CK(cudaStreamSynchronize(st));
        Tile *nt_buf = (Tile *)r->alloc.get(sizeof(Tile) * (size_t)cap, st);
        if (!nt_buf) return fail(QQA_ENOMEM, "tile list allocation failed");
        r->alloc.put(r->d_tiles, st);
        r->d_tiles = nt_buf;
        r->tile_cap = cap;
        drop_graphs(r);  // captured graphs hold the old tile pointer
    }
    if (nt) QQA_CK(cudaMemcpyAsync(r->d_tiles, tiles.data(), sizeof(Tile) * (size_t)nt, cudaMemcpyHostToDevice, st));
    // tensor-core runs: the update kernel's 32-row tiles
    int32_t nt2 = 0;
    if (r->dense_N) {
        std::vector<Tile> t2;
        for (int32_t k = 0; k < r->capacity; ++k) {
            const SlotHost &s = r->slots[k];
            if (!s.active) continue;
            for (int32_t row0 = 0; row0 < s.n; row0 += 32) t2.push_back(Tile{k, row0});
        }
        nt2 = (int32_t)t2.size();
        if (nt2 > r->tile2_cap || (r->tile2_cap > 256 && nt2 < r->tile2_cap / 4)) {
            const int32_t cap = nt2 > r->tile2_cap ? std::max<int32_t>(nt2, 2 * r->tile2_cap) : std::max(2 * nt2, 256);
            QQA_CK(cudaStreamSynchronize(st));
            Tile *buf = (Tile *)r->alloc.get(sizeof(Tile) * (size_t)cap, st);
            if (!buf) return fail(QQA_ENOMEM, "tile list allocation failed");
            r->alloc.put(r->d_tiles2, st);
            r->d_tiles2 = buf;
            r->tile2_cap = cap;
            drop_graphs(r);
        }
        if (nt2) QQA_CK(cudaMemcpyAsync(r->d_tiles2, t2.data(), sizeof(Tile) * (size_t)nt2, cudaMemcpyHostToDevice, st));
    }
    r->num_tiles2 = nt2;
    // long-row work items (one per segment) and the max-clique slots
    std::vector<Tile> hub;
    std::vector<int32_t> cliques;
    for (int32_t k = 0; k < r->capacity; ++k) {
        const SlotHost &s = r->slots[k];
        if (!s.active) continue;
        if (r->h_descs[k].hub_active && !fold)
            for (int32_t q = 0; q < s.prob->nseg; ++q) hub.push_back(Tile{k, q});
        if (s.prob->kind == QQA_MAXCLIQUE) cliques.push_back(k);
    }
    const int32_t nh = (int32_t)hub.size(), nc = (int32_t)cliques.size();
    if (resize_to(nh, r->hub_cap) != r->hub_cap) {
        const int32_t cap = resize_to(nh, r->hub_cap);
        QQA_CK(cudaStreamSynchronize(st));
        Tile *buf = (Tile *)r->alloc.get(sizeof(Tile) * (size_t)cap, st);
        if (!buf) return fail(QQA_ENOMEM, "long-row item list allocation failed");
        r->alloc.put(r->d_hub_items, st);
        r->d_hub_items = buf;
        r->hub_cap = cap;
        drop_graphs(r);
    }
    if (nh) QQA_CK(cudaMemcpyAsync(r->d_hub_items, hub.data(), sizeof(Tile) * (size_t)nh, cudaMemcpyHostToDevice, st));
    if (resize_to(nc, r->clique_cap) != r->clique_cap) {
        const int32_t cap = resize_to(nc, r->clique_cap);
        QQA_CK(cudaStreamSynchronize(st));
        int32_t *buf = (int32_t *)r->alloc.get(sizeof(int32_t) * (size_t)cap, st);
        if (!buf) return fail(QQA_ENOMEM, "clique slot list allocation failed");
        r->alloc.put(r->d_clique_slots, st);
        r->d_clique_slots = buf;
        r->clique_cap = cap;
        drop_graphs(r);
    }
    if (nc)
        QQA_CK(cudaMemcpyAsync(r->d_clique_slots, cliques.data(), sizeof(int32_t) * (size_t)nc, cudaMemcpyHostToDevice,
                               st));
    // the launches of a step depend on these counts: captured graphs are redone when they change
    const int32_t groups = r->hub_fn ? 256 / r->cfg.group_lanes : 1;
    const int32_t hub_grid = nh == 0 ? 0 : (r->dynamic ? r->hub_max_grid : std::min(r->hub_max_grid, (nh + groups - 1) / groups));
    if (hub_grid != r->hub_grid || nc != r->num_clique || seg_items != r->seg_items) drop_graphs(r);
    r->seg_items = seg_items;
    r->hub_grid = hub_grid;
    r->num_hub_items = nh;
    r->num_clique = nc;
    r->kernels_per_step = 1 + (r->upd_fn ? 1 : 0) + (nh ? 1 : 0) + (nc ? 1 : 0);
    // chains: tensor-core runs of several instances with neither long rows nor
    // clique column sums (both need every row of the step done); chain c takes
    // whole instances, in slot order, until it holds its share of the row tiles
    int32_t nch = 1, t0[kMaxChains + 1] = {}, u0[kMaxChains + 1] = {};
    if (r->dense_N && !r->dynamic && nh == 0 && nc == 0 && r->chain_st[0]) {
        int32_t active = 0;
        for (int32_t k = 0; k < r->capacity; ++k) active += r->slots[k].active ? 1 : 0;
        nch = std::max(1, std::min(kChains, active));
        int32_t c = 0, ta = 0, ua = 0;
        for (int32_t k = 0; k < r->capacity; ++k) {
            const SlotHost &s = r->slots[k];
            if (!s.active) continue;
            if (c + 1 < nch && (int64_t)ta * nch >= (int64_t)(c + 1) * nt) {   // one new chain per instance at most
                t0[++c] = ta;
                u0[c] = ua;
            }
            ta += (s.n + r->rows_per_tile - 1) / r->rows_per_tile;
            ua += (s.n + 31) / 32;
        }
        nch = c + 1;
        t0[nch] = nt;
        u0[nch] = nt2;
    }
    bool same = nch == r->nchains;
    for (int32_t c = 0; c <= nch && same; ++c) same = t0[c] == r->chain_t0[c] && u0[c] == r->chain_u0[c];
    if (!same) drop_graphs(r);
    r->nchains = nch;
    for (int32_t c = 0; c <= kMaxChains; ++c) {
        r->chain_t0[c] = c <= nch ? t0[c] : 0;
        r->chain_u0[c] = c <= nch ? u0[c] : 0;
    }
    if (nch > 1) r->kernels_per_step = 2 * nch;   // product and update of each chain
    // second word: the run's replica state (p^t, p^{t+1}, master, m, v) is larger
    // than most of L2, so streaming kernels mark it evict-first
    double state_bytes = 0.0;
    const double per_elem = r->prec == kFP32 ? 16.0 : 12.0;   // p^t, p^{t+1}, m, v (BF16: and the master)
    for (int32_t k = 0; k < r->capacity; ++k)
        if (r->slots[k].active) state_bytes += per_elem * (double)r->slots[k].n * (double)r->slots[k].S_pad;
    int dev = 0, l2 = 0;
    QQA_CK(cudaGetDevice(&dev));
    QQA_CK(cudaDeviceGetAttribute(&l2, cudaDevAttrL2CacheSize, dev));
    r->tile_words[0] = nt;
    r->tile_words[1] = state_bytes > 0.75 * (double)l2 ? 1 : 0;
    r->tile_words[2] = nh;
    r->tile_words[3] = nt2;
    for (int32_t c = 0; c < kMaxChains; ++c) {
        r->tile_words[4 + c] = c < r->nchains ? r->chain_t0[c + 1] - r->chain_t0[c] : 0;
        r->tile_words[4 + kMaxChains + c] = c < r->nchains ? r->chain_u0[c + 1] - r->chain_u0[c] : 0;
    }
    QQA_CK(cudaMemcpyAsync(r->d_num_tiles, r->tile_words, sizeof r->tile_words, cudaMemcpyHostToDevice, st));
    QQA_CK(cudaStreamSynchronize(st));
    r->num_tiles = nt;
    return QQA_OK;
}

static int run_create_hinted(int32_t capacity, int32_t S_max, int32_t precision, const qqa_launch_config *cfg,
                             const qqa_allocator *alloc, void *stream, int staged_hint, int32_t mean_deg,
                             qqa_run **out);

extern "C" int qqa_run_create_empty(int32_t capacity, int32_t S_max, int32_t precision, const qqa_launch_config *cfg,
                                    const qqa_allocator *alloc, void *stream, qqa_run **out)
{
    const int rc = run_create_hinted(capacity, S_max, precision, cfg, alloc, stream, 0, 0, out);
    if (!rc) (*out)->dynamic = true;
    return rc;
}

static int run_create_hinted(int32_t capacity, int32_t S_max, int32_t precision, const qqa_launch_config *cfg,
                             const qqa_allocator *alloc, void *stream, int staged_hint, int32_t mean_deg,
                             qqa_run **out)
{
    if (!out) return fail(QQA_EINVAL, "out is NULL");
    *out = nullptr;
    if (capacity < 1 || capacity > 65535) return fail(QQA_EINVAL, "capacity must be in [1, 65535] (got %d)", capacity);
    if (precision != QQA_FP32 && precision != QQA_BF16) return fail(QQA_EINVAL, "unknown precision %d", precision);
    if (S_max < 1 || S_max > 1024) return fail(QQA_EINVAL, "S_max must be in [1, 1024] (got %d)", S_max);
    cudaStream_t st = (cudaStream_t)stream;
    qqa_run *r = new (std::nothrow) qqa_run();
    if (!r) return fail(QQA_ENOMEM, "host allocation failed");
    r->capacity = capacity;
    r->prec = precision;
    r->vec = S_max == 1 ? 1 : (precision == QQA_FP32 ? 4 : 8);   // one replica: no padding lanes
    r->mean_deg_hint = mean_deg;
    r->S_max = S_max;
    r->S_max_pad = (S_max + r->vec - 1) / r->vec * r->vec;
    r->alloc = Alloc::from(alloc);
    int rc = resolve_config(r, cfg, staged_hint);
    if (rc) { delete r; return rc; }
    r->h_descs.assign(capacity, InstDesc{});
    r->slots.resize(capacity);
    r->d_descs = (InstDesc *)r->alloc.get(sizeof(InstDesc) * (size_t)capacity, st);
    r->d_num_tiles = (int32_t *)r->alloc.get(sizeof r->tile_words, st);
    r->d_status = (RunStatus *)r->alloc.get(sizeof(RunStatus), st);
    if (!r->d_descs || !r->d_num_tiles || !r->d_status) {
        qqa_run_destroy(r);
        return fail(QQA_ENOMEM, "run allocation failed");
    }
    cudaError_t e = cudaMemcpyAsync(r->d_descs, r->h_descs.data(), sizeof(InstDesc) * (size_t)capacity,
                                    cudaMemcpyHostToDevice, st);
    if (e == cudaSuccess) e = cudaMemsetAsync(r->d_num_tiles, 0, sizeof r->tile_words, st);
    if (e == cudaSuccess) e = cudaMemsetAsync(r->d_status, 0, sizeof(RunStatus), st);
    if (e == cudaSuccess) e = cudaStreamCreateWithFlags(&r->cap_stream, cudaStreamNonBlocking);
    if (e == cudaSuccess && r->dense_N) {   // the chains' streams and events
        e = cudaEventCreateWithFlags(&r->ev_fork, cudaEventDisableTiming);
        for (int c = 0; c < kChains - 1 && e == cudaSuccess; ++c) {
            e = cudaStreamCreateWithFlags(&r->chain_st[c], cudaStreamNonBlocking);
            if (e == cudaSuccess) e = cudaEventCreateWithFlags(&r->ev_join[c], cudaEventDisableTiming);
        }
    }
    if (e == cudaSuccess) e = cudaStreamSynchronize(st);
    if (e != cudaSuccess) {
        qqa_run_destroy(r);
        return fail(QQA_ECUDA, "run setup: %s", cudaGetErrorString(e));
    }
    *out = r;
    return QQA_OK;
}

static int check_params(const qqa_params *p, int32_t S_max, int32_t prec)
{
    if (!p) return fail(QQA_EINVAL, "params is NULL");
    if (p->S < 1 || p->S > S_max) return fail(QQA_EINVAL, "S = %d outside [1, %d]", p->S, S_max);
    if (p->steps < 1) return fail(QQA_EINVAL, "steps must be >= 1");
    if (p->round_every < 0) return fail(QQA_EINVAL, "round_every must be >= 0");
    if (p->a_ent < 2 || p->a_ent > 8 || p->a_ent % 2) return fail(QQA_EINVAL, "a_ent must be 2, 4, 6 or 8");
    if (!(p->lr > 0.0f) || !std::isfinite(p->lr)) return fail(QQA_EINVAL, "lr must be positive and finite");
    if (!(p->beta1 >= 0.5f && p->beta1 < 1.0f) || !(p->beta2 >= 0.5f && p->beta2 < 1.0f))
        return fail(QQA_EINVAL, "beta1, beta2 must lie in [0.5, 1)");
    if (!(p->adam_eps > 0.0f) || !(p->comm_eps >= 0.0f) || !(p->temperature >= 0.0f) || !(p->weight_decay >= 0.0f))
        return fail(QQA_EINVAL, "adam_eps > 0 and comm_eps, temperature, weight_decay >= 0 required");
    if (!std::isfinite(p->gamma_min) || !std::isfinite(p->gamma_max) || !std::isfinite(p->alpha_comm) ||
        !std::isfinite(p->lambda))
        return fail(QQA_EINVAL, "gamma, alpha_comm and lambda must be finite");
    if (p->alpha_comm != 0.0f && !(p->comm_eps > 0.0f)) return fail(QQA_EINVAL, "alpha_comm != 0 needs comm_eps > 0");
    if (p->precision != prec) return fail(QQA_EINVAL, "instance precision %d differs from the run's %d", p->precision, prec);
    return QQA_OK;
}

static PFN_cuTensorMapEncodeTiled_v12000 tensor_map_encoder()
{
    static PFN_cuTensorMapEncodeTiled_v12000 fn = nullptr;
    static std::once_flag once;
    std::call_once(once, [] {
        cudaDriverEntryPointQueryResult q;
        void *p = nullptr;
        if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault, &q) ==
                cudaSuccess &&
            q == cudaDriverEntryPointSuccess)
            fn = reinterpret_cast<PFN_cuTensorMapEncodeTiled_v12000>(p);
        (void)cudaGetLastError();
    });
    return fn;
}

// A 2-D fp16 tensor map with 128-byte swizzle (shared with color.cu): `outer`
// rows of `inner` elements, rows `row_bytes` apart, box of box_inner x
// box_outer. Returns 0 on success.
namespace qqa {
int encode_tmap_f16_2d(void *map_out, const void *base, uint64_t inner, uint64_t outer, uint64_t row_bytes,
                       uint32_t box_inner, uint32_t box_outer)
{
    PFN_cuTensorMapEncodeTiled_v12000 enc = tensor_map_encoder();
    if (!enc) return -1;
    const cuuint32_t es[2] = {1, 1};
    const cuuint64_t dims[2] = {(cuuint64_t)inner, (cuuint64_t)outer}, str[1] = {(cuuint64_t)row_bytes};
    const cuuint32_t box[2] = {box_inner, box_outer};
    const CUresult cr = enc(reinterpret_cast<CUtensorMap *>(map_out), CU_TENSOR_MAP_DATA_TYPE_FLOAT16, 2,
                            const_cast<void *>(base), dims, str, box, es, CU_TENSOR_MAP_INTERLEAVE_NONE,
                            CU_TENSOR_MAP_SWIZZLE_128B, CU_TENSOR_MAP_L2_PROMOTION_L2_128B,
                            CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
    return cr == CUDA_SUCCESS ? 0 : (int)cr;
}
}  // namespace qqa

// Adjacency in fp16, state planes, and the five TMA tensor maps of a dense slot.
static int setup_dense_slot(qqa_run *r, int32_t k, InstDesc &d, std::vector<void *> &dev, cudaStream_t st)
{
    const int N = r->dense_N;
    const int64_t n_pad = (d.n + 127) / 128 * 128;
    const size_t a_bytes = (size_t)n_pad * n_pad * 2, x_bytes = (size_t)4 * N * n_pad * 2;
    d.n_pad = (int32_t)n_pad;
    d.dense_N = N;
    d.dense_A = (uint16_t *)r->alloc.get(a_bytes, st);
    d.dense_XT = (uint16_t *)r->alloc.get(x_bytes, st);
    d.dense_Y = (float *)r->alloc.get((size_t)d.n * r->slots[k].S_pad * sizeof(float), st);
    void *tm = r->alloc.get(5 * sizeof(CUtensorMap), st);
    if (d.dense_A) dev.push_back(d.dense_A);
    if (d.dense_XT) dev.push_back(d.dense_XT);
    if (d.dense_Y) dev.push_back(d.dense_Y);
    if (tm) dev.push_back(tm);
    if (!d.dense_A || !d.dense_XT || !d.dense_Y || !tm)
        return fail(QQA_ENOMEM, "dense adjacency of %lld x %lld fp16 does not fit", (long long)n_pad, (long long)n_pad);
    // unit-weight graphs: adjacency and rounded replicas as bitsets, so the
    // evaluation counts by popcount
    d.dense_Abits = nullptr;
    d.dense_xbits = nullptr;
    size_t ab_bytes = 0;
    if (!d.w) {
        ab_bytes = (size_t)n_pad * (size_t)(n_pad / 32) * 4;
        const size_t xb_bytes = (size_t)((r->slots[k].S_pad + 31) / 32 * 32) * (size_t)(n_pad / 32) * 4;
        d.dense_Abits = (uint32_t *)r->alloc.get(ab_bytes, st);
        d.dense_xbits = (uint32_t *)r->alloc.get(xb_bytes, st);
        if (d.dense_Abits) dev.push_back(d.dense_Abits);
        if (d.dense_xbits) dev.push_back(d.dense_xbits);
        if (!d.dense_Abits || !d.dense_xbits) return fail(QQA_ENOMEM, "dense adjacency bitsets do not fit");
        QQA_CK(cudaMemsetAsync(d.dense_Abits, 0, ab_bytes, st));
    }
    d.dense_tmaps = tm;
    PFN_cuTensorMapEncodeTiled_v12000 enc = tensor_map_encoder();
    if (!enc) return fail(QQA_ECUDA, "cuTensorMapEncodeTiled is not available");
    alignas(64) CUtensorMap maps[5];
    const cuuint32_t es[2] = {1, 1};
    const cuuint64_t adims[2] = {(cuuint64_t)n_pad, (cuuint64_t)n_pad}, astr[1] = {(cuuint64_t)n_pad * 2};
    const cuuint32_t abox[2] = {64, 128};
    CUresult cr = enc(&maps[0], CU_TENSOR_MAP_DATA_TYPE_FLOAT16, 2, d.dense_A, adims, astr, abox, es,
                      CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_128B, CU_TENSOR_MAP_L2_PROMOTION_L2_128B,
                      CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
    const cuuint64_t xdims[2] = {(cuuint64_t)n_pad, (cuuint64_t)N}, xstr[1] = {(cuuint64_t)n_pad * 2};
    const cuuint32_t xbox[2] = {64, (cuuint32_t)N};
    for (int p = 0; p < 4 && cr == CUDA_SUCCESS; ++p)
        cr = enc(&maps[1 + p], CU_TENSOR_MAP_DATA_TYPE_FLOAT16, 2, d.dense_XT + (size_t)p * N * n_pad, xdims, xstr,
                 xbox, es, CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_128B,
                 CU_TENSOR_MAP_L2_PROMOTION_L2_128B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
    if (cr != CUDA_SUCCESS) return fail(QQA_ECUDA, "tensor map encoding failed (%d)", (int)cr);
    QQA_CK(cudaMemsetAsync(d.dense_A, 0, a_bytes, st));
    QQA_CK(cudaMemsetAsync(d.dense_XT, 0, x_bytes, st));
    QQA_CK(cudaMemcpyAsync(tm, maps, sizeof maps, cudaMemcpyHostToDevice, st));
    QQA_CK(cudaStreamSynchronize(st));
    return QQA_OK;
}

static void free_slot(qqa_run *r, int32_t k, cudaStream_t st)
{
    SlotHost &s = r->slots[k];
    for (void *p : s.dev) r->alloc.put(p, st);
    s = SlotHost{};
    r->h_descs[k] = InstDesc{};
}

// Device memory of one slot: every buffer is carved out of one allocation
// (256-byte aligned pieces), so adding an instance costs one allocator call.
struct SlotLayout {
    size_t X[2], master, m, v, colsum, seg_part, seg_cnt, bits, counts, res_obj, res_viol, res_feas, res_energy,
        res_meta, res_bestx, hist_best, hist_step, scal, total;
};

static const size_t kNone = ~(size_t)0;

static SlotLayout slot_layout(int32_t n, int32_t S_pad, int32_t W, int32_t hist_cap, int32_t prec, bool clique,
                              int32_t nseg, int32_t nlong)
{
    SlotLayout L{};
    size_t off = 0;
    auto take = [&](size_t bytes) {
        const size_t o = off;
        off += (std::max<size_t>(bytes, 16) + 255) & ~(size_t)255;
        return o;
    };
    const size_t elems = (size_t)n * S_pad, tb = prec == kFP32 ? 4 : 2;
    L.X[0] = take(elems * tb);
    L.X[1] = take(elems * tb);
    L.master = prec == kBF16 ? take(elems * 4) : kNone;
    L.m = take(elems * tb);
    L.v = take(elems * tb);
    L.colsum = clique ? take((size_t)S_pad * 4) : kNone;
    L.seg_part = nseg > 0 ? take((size_t)nseg * S_pad * 4) : kNone;
    L.seg_cnt = nseg > 0 ? take((size_t)nlong * 4) : kNone;
    L.bits = take((size_t)n * W * 4);
    L.counts = take(3 * (size_t)S_pad * 8);
    L.res_obj = take((size_t)S_pad * 8);
    L.res_viol = take((size_t)S_pad * 8);
    L.res_feas = take((size_t)S_pad);
    L.res_energy = take((size_t)S_pad * 8);
    L.res_meta = take(4 * 4);
    L.res_bestx = take((size_t)((n + 31) / 32) * 4);
    L.hist_best = take((size_t)hist_cap * 8);
    L.hist_step = take((size_t)hist_cap * 4);
    L.scal = take((size_t)kMaxChunk * sizeof(float4));
    L.total = off;
    return L;
}

namespace qqa {
// Device bytes one request takes when it is added to a run of a gathering
// step kernel: the graph (CSR, weights, long-row tables) and the slot's
// carved state, each allocation rounded up to 512 bytes (the granule of the
// usual allocators), plus its share of the run's work lists (at most one tile
// per row and one item per long-row segment, in lists whose capacity stays
// within four times their entries: they double when full and halve below a
// quarter).
int64_t request_device_bytes(int32_t kind, int32_t n, const int32_t *row_ptr, bool weighted, const qqa_params *prm)
{
    auto g512 = [](int64_t b) { return (std::max<int64_t>(b, 16) + 511) / 512 * 512; };
    const int64_t nnz = row_ptr[n];
    const int32_t thr = long_row_threshold(n, nnz);
    int32_t nlong = 0, nseg = 0;
    for (int32_t i = 0; i < n; ++i) {
        const int32_t deg = row_ptr[i + 1] - row_ptr[i];
        if (deg > thr) { ++nlong; nseg += (deg + kSegLen - 1) / kSegLen; }
    }
    const int32_t vec = prm->precision == QQA_FP32 ? 4 : 8;
    const int32_t S_pad = prm->S == 1 ? 1 : (prm->S + vec - 1) / vec * vec;
    const int32_t hist_cap = (prm->round_every > 0 ? prm->steps / prm->round_every : 0) + 2;
    int64_t b = g512(4 * ((int64_t)n + 1)) + g512(4 * nnz) + (weighted ? g512(4 * nnz) : 0);
    if (nlong) b += g512(4 * (int64_t)nlong) + g512(4 * ((int64_t)nlong + 1)) + g512(4 * (int64_t)nseg);
    const SlotLayout L = slot_layout(n, S_pad, (prm->S + 31) / 32, hist_cap, prm->precision, kind == QQA_MAXCLIQUE,
                                     nseg, nlong);
    b += g512((int64_t)L.total);
    b += 32 * ((int64_t)n + nseg);   // tile and segment records (lists hold at most 4x their entries)
    return b;
}
}  // namespace qqa

// First half of adding an instance: a free slot, its device memory and its
// host-side descriptor. Nothing is launched.
static int slot_setup(qqa_run *r, const qqa_problem *prob, const qqa_params *prm, cudaStream_t st, int32_t *slot_out)
{
    if (!r || !prob) return fail(QQA_EINVAL, "run or problem is NULL");
    int rc = check_params(prm, r->S_max, r->prec);
    if (rc) return rc;
    int32_t k = -1;
    for (int32_t i = 0; i < r->capacity; ++i)
        if (!r->slots[i].active) { k = i; break; }
    if (k < 0) return fail(QQA_EBUSY, "no free slot (capacity %d)", r->capacity);

    SlotHost &s = r->slots[k];
    s = SlotHost{};
    s.prob = prob;
    s.prm = *prm;
    s.n = prob->n;
    s.S = prm->S;
    s.S_pad = (prm->S + r->vec - 1) / r->vec * r->vec;
    s.W = (prm->S + 31) / 32;
    s.K = prm->steps;
    s.hist_cap = (prm->round_every > 0 ? prm->steps / prm->round_every : 0) + 2;
    // long rows: the evaluation always splits them; the gather step kernels
    // leave them to segment work items (partial sums and counters per slot)
    const bool hubs = r->hub_fn != nullptr && prob->nlong > 0;
    const SlotLayout L = slot_layout(s.n, s.S_pad, s.W, s.hist_cap, r->prec, prob->kind == QQA_MAXCLIQUE,
                                     hubs ? prob->nseg : 0, prob->nlong);
    unsigned char *base = (unsigned char *)r->alloc.get(L.total, st);
    if (!base) return fail(QQA_ENOMEM, "device allocation of %zu bytes for instance state failed (n=%d, S=%d)",
                           L.total, s.n, s.S);
    s.dev.push_back(base);
    if ((uintptr_t)base & 15u) {
        free_slot(r, k, st);
        return fail(QQA_EINVAL, "the allocator returned state memory that is not 16-byte aligned");
    }
    auto at = [&](size_t off) -> void * { return off == kNone ? nullptr : (void *)(base + off); };
    InstDesc d{};
    d.row_ptr = prob->row_ptr;
    d.col = prob->col;
    d.w = prob->w;
    d.X[0] = at(L.X[0]);
    d.X[1] = at(L.X[1]);
    d.master = (float *)at(L.master);
    d.m = at(L.m);
    d.v = at(L.v);
    d.colsum = (float *)at(L.colsum);
    d.long_thresh = prob->nlong > 0 ? prob->long_thresh : 0x7fffffff;
    d.hub_active = hubs ? 1 : 0;
    d.nlong = prob->nlong;
    d.nseg = prob->nseg;
    d.long_rows = prob->long_rows;
    d.seg_ptr = prob->seg_ptr;
    d.seg_row = prob->seg_row;
    d.seg_part = (float *)at(L.seg_part);
    d.seg_cnt = (uint32_t *)at(L.seg_cnt);
    d.grad_dbg = nullptr;
    d.bits = (uint32_t *)at(L.bits);
    d.counts = (unsigned long long *)at(L.counts);
    d.res_obj = (long long *)at(L.res_obj);
    d.res_viol = (long long *)at(L.res_viol);
    d.res_feas = (uint8_t *)at(L.res_feas);
    d.res_energy = (double *)at(L.res_energy);
    d.res_meta = (int32_t *)at(L.res_meta);
    d.res_bestx = (uint32_t *)at(L.res_bestx);
    d.hist_best = (long long *)at(L.hist_best);
    d.hist_step = (int32_t *)at(L.hist_step);
    d.scal = (float4 *)at(L.scal);
    if (r->dense_N) {
        if (prob->max_abs_w > 2048) {
            free_slot(r, k, st);
            return fail(QQA_EINVAL, "edge weights above 2048 are not exact in the fp16 adjacency of the dense step");
        }
        d.n = s.n;
        const int drc = setup_dense_slot(r, k, d, s.dev, st);
        if (drc) {
            const std::string msg = g_last_error;
            free_slot(r, k, st);
            return fail(drc, "%s", msg.c_str());
        }
    }
    d.n = s.n;
    d.S = s.S;
    d.S_pad = s.S_pad;
    d.W = s.W;
    d.kind = prob->kind;
    d.a_ent = prm->a_ent;
    d.t = 0;
    d.K = prm->steps;
    d.active = 1;
    d.hist_cap = s.hist_cap;
    d.last_eval_t = -1;
    d.lr = prm->lr;
    d.wd = prm->weight_decay;
    d.b1 = prm->beta1;
    d.b2 = prm->beta2;
    d.adam_eps = prm->adam_eps;
    d.gmin = prm->gamma_min;
    d.gmax = prm->gamma_max;
    d.alpha = prm->alpha_comm;
    d.comm_eps = prm->comm_eps;
    d.noise_scale = (float)std::sqrt(2.0 * (double)prm->lr * (double)prm->temperature);
    d.lambda = prm->lambda;
    d.decay = 1.0f - prm->lr * prm->weight_decay;
    d.seed_lo = (uint32_t)(prm->seed & 0xffffffffu);
    d.seed_hi = (uint32_t)(prm->seed >> 32);
    r->h_descs[k] = d;
    s.active = true;
    s.obj.assign(s.S, 0);
    s.viol.assign(s.S, 0);
    s.feas.assign(s.S, 0);
    s.energy.assign(s.S, 0.0);
    cudaError_t e = cudaMemsetAsync(d.res_meta, 0, 16, st);
    if (e == cudaSuccess && hubs) e = cudaMemsetAsync(d.seg_cnt, 0, (size_t)prob->nlong * 4, st);
    if (e != cudaSuccess) { free_slot(r, k, st); return fail(QQA_ECUDA, "memset: %s", cudaGetErrorString(e)); }
    *slot_out = k;
    return QQA_OK;
}

// Second half: the initial draw (and the max-clique column sums, the
// tensor-core adjacency and planes) of a slot whose descriptor is on the device.
static int slot_start(qqa_run *r, int32_t k, cudaStream_t st)
{
    const SlotHost &s = r->slots[k];
    launch_init(r->d_descs, k, s.n, s.S_pad, r->prec, st);
    g_launches += 1;
    if (s.prob->kind == QQA_MAXCLIQUE) {
        launch_colsum(r->d_descs, nullptr, 1, k, s.S_pad, r->prec, 0, 0, st);
        g_launches += 1;
    }
    if (r->dense_N) {
        launch_dense_adjacency(r->d_descs, k, s.n, st);
        launch_dense_planes(r->d_descs, k, s.n, s.S_pad, st);
        g_launches += 2;
    }
    QQA_CK_LAUNCH("init");
    return QQA_OK;
}

extern "C" int qqa_run_add(qqa_run *r, const qqa_problem *prob, const qqa_params *prm, void *stream, int32_t *slot_out)
{
    cudaStream_t st = (cudaStream_t)stream;
    int32_t k = -1;
    int rc = slot_setup(r, prob, prm, st, &k);
    if (rc) return rc;
    rc = upload_desc(r, k, st);
    if (!rc) rc = slot_start(r, k, st);
    if (rc) { free_slot(r, k, st); return rc; }
    rc = rebuild_tiles(r, st);
    if (rc) {   // no room for the grown tile list: undo the add, keep the other slots running
        const std::string msg = g_last_error;
        r->h_descs[k].active = 0;
        r->slots[k].active = false;
        (void)upload_desc(r, k, st);
        cudaStreamSynchronize(st);
        free_slot(r, k, st);
        (void)rebuild_tiles(r, st);
        return fail(rc, "%s", msg.c_str());
    }
    if (slot_out) *slot_out = k;
    return QQA_OK;
}

extern "C" int qqa_run_reset(qqa_run *r, int32_t slot, uint64_t seed, void *stream)
{
    if (!r) return fail(QQA_EINVAL, "run is NULL");
    if (slot < -1 || slot >= r->capacity || (slot >= 0 && !r->slots[slot].active))
        return fail(QQA_EINVAL, "bad slot %d", slot);
    cudaStream_t st = (cudaStream_t)stream;
    bool any = false;
    for (int32_t k = 0; k < r->capacity; ++k) {
        if ((slot >= 0 && k != slot) || !r->slots[k].active) continue;
        SlotHost &s = r->slots[k];
        s.t = 0;
        s.last_eval_t = -1;
        s.eval_count = 0;
        s.prm.seed = seed;
        r->h_descs[k].seed_lo = (uint32_t)(seed & 0xffffffffu);
        r->h_descs[k].seed_hi = (uint32_t)(seed >> 32);
        any = true;
    }
    if (!any) return QQA_OK;
    // one upload of the whole table (reset slots changed t, seed, eval marker)
    for (int32_t k = 0; k < r->capacity; ++k) {
        r->h_descs[k].t = r->slots[k].t;
        r->h_descs[k].last_eval_t = r->slots[k].last_eval_t;
    }
    // (a copy from pageable host memory is staged before the call returns, so
    // the table may change afterwards; the host does not wait for the device
    // here, and a caller can queue several anneals ahead)
    QQA_CK(cudaMemcpyAsync(r->d_descs, r->h_descs.data(), sizeof(InstDesc) * (size_t)r->capacity,
                           cudaMemcpyHostToDevice, st));
    for (int32_t k = 0; k < r->capacity; ++k) {
        if ((slot >= 0 && k != slot) || !r->slots[k].active) continue;
        const SlotHost &s = r->slots[k];
        QQA_CK(cudaMemsetAsync(r->h_descs[k].res_meta, 0, 16, st));
        if (r->h_descs[k].seg_cnt) QQA_CK(cudaMemsetAsync(r->h_descs[k].seg_cnt, 0, (size_t)s.prob->nlong * 4, st));
        launch_init(r->d_descs, k, s.n, s.S_pad, r->prec, st);
        g_launches += 1;
        if (s.prob->kind == QQA_MAXCLIQUE) {
            launch_colsum(r->d_descs, nullptr, 1, k, s.S_pad, r->prec, 0, 0, st);
            g_launches += 1;
        }
        if (r->dense_N) {
            launch_dense_planes(r->d_descs, k, s.n, s.S_pad, st);
            g_launches += 1;
        }
    }
    QQA_CK_LAUNCH("reset");
    return QQA_OK;
}

extern "C" int qqa_run_remove(qqa_run *r, int32_t k, void *stream)
{
    if (!r || k < 0 || k >= r->capacity || !r->slots[k].active) return fail(QQA_EINVAL, "bad slot %d", k);
    cudaStream_t st = (cudaStream_t)stream;
    r->h_descs[k].active = 0;
    int rc = upload_desc(r, k, st);
    if (rc) return rc;
    QQA_CK(cudaStreamSynchronize(st));
    free_slot(r, k, st);
    return rebuild_tiles(r, st);
}

extern "C" int qqa_run_create(qqa_problem *const *problems, const qqa_params *params, int32_t count,
                              const qqa_launch_config *cfg, const qqa_allocator *alloc, void *stream, qqa_run **out)
{
    if (!problems || !params || count < 1) return fail(QQA_EINVAL, "need count >= 1 problems and params");
    int32_t S_max = 1;
    for (int32_t k = 0; k < count; ++k) {
        if (!problems[k]) return fail(QQA_EINVAL, "problem %d is NULL", k);
        S_max = std::max(S_max, params[k].S);
    }
    if (S_max > 1024) return fail(QQA_EINVAL, "S = %d exceeds 1024", S_max);
    // Auto kernel choice: staging pays when gathering every neighbour row from
    // L2 would move more than twice the bytes of streaming each block's span
    // of the state once (64-row blocks, the span taken as the whole graph).
    double gather_rows = 0.0, staged_rows = 0.0;
    for (int32_t k = 0; k < count; ++k) {
        gather_rows += (double)problems[k]->nnz;
        staged_rows += (double)((problems[k]->n + 63) / 64) * (double)problems[k]->n;
    }
    // (measured on GB300: the staged kernel does not yet beat the direct one,
    // so auto keeps the direct kernel until it does)
    const int staged_hint = (gather_rows > 2.0 * staged_rows && kAutoStaged) ? 1 : 0;
    double nodes = 0.0;
    for (int32_t k = 0; k < count; ++k) nodes += (double)problems[k]->n;
    const int32_t mean_deg = (int32_t)std::min(1.0e9, std::ceil(gather_rows / std::max(nodes, 1.0)));
    qqa_run *r = nullptr;
    int rc = run_create_hinted(count, S_max, params[0].precision, cfg, alloc, stream, staged_hint, mean_deg, &r);
    if (rc) return rc;
    // every slot set up first, then one descriptor upload, the initial draws
    // and one tile list (slot k = problem k)
    cudaStream_t st = (cudaStream_t)stream;
    for (int32_t k = 0; k < count && !rc; ++k) {
        int32_t slot = -1;
        rc = slot_setup(r, problems[k], &params[k], st, &slot);
        if (rc) {
            std::string msg = g_last_error;
            qqa_run_destroy(r);
            return fail(rc, "instance %d: %s", k, msg.c_str());
        }
    }
    cudaError_t e = cudaMemcpyAsync(r->d_descs, r->h_descs.data(), sizeof(InstDesc) * (size_t)count,
                                    cudaMemcpyHostToDevice, st);
    if (e != cudaSuccess) rc = fail(QQA_ECUDA, "descriptor upload: %s", cudaGetErrorString(e));
    for (int32_t k = 0; k < count && !rc; ++k) rc = slot_start(r, k, st);
    if (!rc) rc = rebuild_tiles(r, st);
    if (rc) {
        std::string msg = g_last_error;
        qqa_run_destroy(r);
        return fail(rc, "%s", msg.c_str());
    }
    *out = r;
    return QQA_OK;
}

extern "C" void qqa_run_destroy(qqa_run *r)
{
    if (!r) return;
    cudaDeviceSynchronize();
    drop_graphs(r);
    for (int32_t k = 0; k < (int32_t)r->slots.size(); ++k)
        if (r->slots[k].active) free_slot(r, k, 0);
    r->alloc.put(r->d_descs, 0);
    r->alloc.put(r->d_tiles, 0);
    r->alloc.put(r->d_hub_items, 0);
    r->alloc.put(r->d_tiles2, 0);
    r->alloc.put(r->d_clique_slots, 0);
    r->alloc.put(r->d_num_tiles, 0);
    r->alloc.put(r->d_status, 0);
    r->alloc.put(r->d_scratch, 0);
    if (r->cap_stream) cudaStreamDestroy(r->cap_stream);
    if (r->ev_fork) cudaEventDestroy(r->ev_fork);
    for (int c = 0; c < kMaxChains; ++c) {
        if (r->chain_st[c]) cudaStreamDestroy(r->chain_st[c]);
        if (r->ev_join[c]) cudaEventDestroy(r->ev_join[c]);
    }
    delete r;
}

extern "C" int qqa_run_config(const qqa_run *r, qqa_launch_config *out)
{
    if (!r || !out) return fail(QQA_EINVAL, "NULL argument");
    *out = r->cfg;
    return QQA_OK;
}

// ------------------------------------------------------------------- steps
// The steps of a chunk for a chained tensor-core run: chain 0 on st, chain c
// on the run's stream c - 1 (forked from st and joined back at the end). Each
// chain's steps depend only on its own previous step.
static int launch_chains(qqa_run *r, int32_t chunk, cudaStream_t st)
{
    const int32_t nch = r->nchains;
    launch_prepare(r->d_descs, r->capacity, chunk, st);
    QQA_CK(cudaEventRecord(r->ev_fork, st));
    for (int32_t c = 1; c < nch; ++c) QQA_CK(cudaStreamWaitEvent(r->chain_st[c - 1], r->ev_fork, 0));
    for (int32_t i = 0; i < chunk; ++i)
        for (int32_t c = 0; c < nch; ++c) {
            cudaStream_t s = c == 0 ? st : r->chain_st[c - 1];
            const int32_t nt = r->chain_t0[c + 1] - r->chain_t0[c], nu = r->chain_u0[c + 1] - r->chain_u0[c];
            r->step_fn<<<std::max(1, std::min(r->max_grid, nt)), r->cfg.block_threads, r->smem, s>>>(
                r->d_descs, r->d_tiles + r->chain_t0[c], r->d_num_tiles + 4 + c, r->d_status, i);
            r->upd_fn<<<std::max(1, std::min(r->upd_max_grid, nu)), r->upd_block, r->upd_smem, s>>>(
                r->d_descs, r->d_tiles2 + r->chain_u0[c], r->d_num_tiles + 4 + kMaxChains + c, r->d_status, i,
                r->upd_ld);
        }
    for (int32_t c = 1; c < nch; ++c) {
        QQA_CK(cudaEventRecord(r->ev_join[c - 1], r->chain_st[c - 1]));
        QQA_CK(cudaStreamWaitEvent(st, r->ev_join[c - 1], 0));
    }
    launch_advance(r->d_descs, r->capacity, chunk, st);
    QQA_CK_LAUNCH("step");
    return QQA_OK;
}

static int launch_step_chunk(qqa_run *r, int32_t chunk, int32_t grid, cudaStream_t st)
{
    if (r->nchains > 1) return launch_chains(r, chunk, st);
    launch_prepare(r->d_descs, r->capacity, chunk, st);
    for (int32_t i = 0; i < chunk; ++i) {
        if (r->tiled_fn)
            r->tiled_fn<<<grid, r->cfg.block_threads, r->smem, st>>>(r->d_descs, r->d_tiles, r->d_num_tiles,
                                                                     r->d_status, i, r->chunk_rows, r->buf_elems);
        else if (r->pipe_fn)
            (r->seg_items ? r->pipe_seg_fn : r->pipe_fn)<<<grid, r->cfg.block_threads, r->smem, st>>>(
                r->d_descs, r->d_tiles, r->d_num_tiles,
                                                                    r->d_status, i, r->pipe_buf);
        else
            r->step_fn<<<grid, r->cfg.block_threads, r->smem, st>>>(r->d_descs, r->d_tiles, r->d_num_tiles,
                                                                    r->d_status, i);
        if (r->upd_fn) {   // tensor-core step: the update of every row after the product
            const int32_t g2 = r->dynamic ? r->upd_max_grid : std::max(1, std::min(r->upd_max_grid, r->num_tiles2));
            r->upd_fn<<<g2, r->upd_block, r->upd_smem, st>>>(r->d_descs, r->d_tiles2, r->d_num_tiles + 3, r->d_status,
                                                             i, r->upd_ld);
        }
        if (r->num_hub_items > 0)   // long rows of the same step (disjoint rows, same p^t)
            r->hub_fn<<<r->hub_grid, 256, 0, st>>>(r->d_descs, r->d_hub_items, r->d_num_tiles + 2, r->d_status, i);
        if (r->num_clique > 0)      // column sums of p^{t+1} for the next step's Eq. 24 term
            launch_colsum(r->d_descs, r->d_clique_slots, r->num_clique, 0, r->S_max_pad, r->prec, i, 1, st);
    }
    launch_advance(r->d_descs, r->capacity, chunk, st);
    QQA_CK_LAUNCH("step");
    return QQA_OK;
}

static int get_graph(qqa_run *r, int32_t chunk, int32_t grid, cudaGraphExec_t *exec)
{
    auto key = std::make_pair(chunk, grid);
    auto it = r->graphs.find(key);
    if (it != r->graphs.end()) { *exec = it->second; return QQA_OK; }
    cudaGraph_t g = nullptr;
    QQA_CK(cudaStreamBeginCapture(r->cap_stream, cudaStreamCaptureModeThreadLocal));
    int rc = launch_step_chunk(r, chunk, grid, r->cap_stream);
    cudaError_t e = cudaStreamEndCapture(r->cap_stream, &g);
    if (rc) { if (g) cudaGraphDestroy(g); return rc; }
    if (e != cudaSuccess) return fail(QQA_ECUDA, "graph capture: %s", cudaGetErrorString(e));
    cudaGraphExec_t ge = nullptr;
    e = cudaGraphInstantiate(&ge, g, 0);
    cudaGraphDestroy(g);
    if (e != cudaSuccess) return fail(QQA_ECUDA, "graph instantiate: %s", cudaGetErrorString(e));
    r->graphs[key] = ge;
    *exec = ge;
    return QQA_OK;
}

static const int32_t kGraphChunk = 50;

extern "C" int qqa_run_steps(qqa_run *r, int32_t nsteps, void *stream)
{
    if (!r) return fail(QQA_EINVAL, "run is NULL");
    if (nsteps < 0) return fail(QQA_EINVAL, "nsteps < 0");
    if (nsteps == 0 || r->num_tiles == 0) return QQA_OK;
    cudaStream_t st = (cudaStream_t)stream;
    const int32_t grid = r->dynamic ? r->max_grid : std::min(r->max_grid, r->num_tiles);
    int32_t left = nsteps;
    while (left > 0) {
        const int32_t chunk = std::min(left, kGraphChunk);
        if (r->cfg.use_graphs) {
            cudaGraphExec_t ge = nullptr;
            int rc = get_graph(r, chunk, grid, &ge);
            if (rc) return rc;
            QQA_CK(cudaGraphLaunch(ge, st));
        } else {
            int rc = launch_step_chunk(r, chunk, grid, st);
            if (rc) return rc;
        }
        g_launches += (unsigned long long)chunk * r->kernels_per_step + 2;
        for (auto &s : r->slots)
            if (s.active) s.t = std::min(s.t + chunk, s.K);
        left -= chunk;
    }
    return QQA_OK;
}

// -------------------------------------------------------------------- eval
extern "C" int qqa_run_eval(qqa_run *r, void *stream)
{
    if (!r) return fail(QQA_EINVAL, "run is NULL");
    if (r->num_tiles == 0) return QQA_OK;
    cudaStream_t st = (cudaStream_t)stream;
    int32_t n_max = 0, seg_max = 0;
    int64_t total_rows = 0;
    for (const auto &s : r->slots)
        if (s.active) {
            n_max = std::max(n_max, s.n);
            seg_max = std::max(seg_max, s.prob->nseg);
            total_rows += s.n;
        }
    launch_eval(r->d_descs, r->capacity, n_max, total_rows, r->S_max_pad, r->prec, r->dense_N > 0, seg_max, st);
    g_launches += r->dense_N > 0 ? 7 : 5;
    QQA_CK_LAUNCH("eval");
    for (auto &s : r->slots)
        if (s.active && s.t != s.last_eval_t) s.last_eval_t = s.t;
    return QQA_OK;
}

extern "C" int qqa_run_sync(qqa_run *r, void *stream)
{
    if (!r) return fail(QQA_EINVAL, "run is NULL");
    cudaStream_t st = (cudaStream_t)stream;
    QQA_CK(cudaStreamSynchronize(st));
    for (int32_t k = 0; k < r->capacity; ++k) {
        SlotHost &s = r->slots[k];
        if (!s.active) continue;
        const InstDesc &d = r->h_descs[k];
        int32_t meta[4] = {0, 0, 0, 0};
        QQA_CK(cudaMemcpy(meta, d.res_meta, sizeof meta, cudaMemcpyDeviceToHost));
        if (meta[2] == 0) continue;  // never evaluated
        QQA_CK(cudaMemcpy(s.obj.data(), d.res_obj, sizeof(long long) * s.S, cudaMemcpyDeviceToHost));
        QQA_CK(cudaMemcpy(s.viol.data(), d.res_viol, sizeof(long long) * s.S, cudaMemcpyDeviceToHost));
        QQA_CK(cudaMemcpy(s.feas.data(), d.res_feas, s.S, cudaMemcpyDeviceToHost));
        QQA_CK(cudaMemcpy(s.energy.data(), d.res_energy, sizeof(double) * s.S, cudaMemcpyDeviceToHost));
        s.best = meta[0];
        s.eval_step = meta[1];
        s.eval_count = meta[2];
    }
    RunStatus stt{};
    QQA_CK(cudaMemcpy(&stt, r->d_status, sizeof stt, cudaMemcpyDeviceToHost));
    if (stt.timeouts)
        return fail(QQA_ETIMEOUT, "%llu staged copies did not arrive within the wait limit", stt.timeouts);
    if (stt.nonfinite) return fail(QQA_ENONFINITE, "%llu non-finite gradient/state values were produced", stt.nonfinite);
    return QQA_OK;
}

extern "C" int qqa_run_result(const qqa_run *r, int32_t k, int64_t *obj, int64_t *viol, uint8_t *feasible,
                              double *energy, int32_t *best_s, uint32_t *best_x, int32_t *step)
{
    if (!r || k < 0 || k >= r->capacity || !r->slots[k].active) return fail(QQA_EINVAL, "bad slot %d", k);
    const SlotHost &s = r->slots[k];
    if (s.eval_count == 0) return fail(QQA_EBUSY, "slot %d has no synchronised evaluation", k);
    if (obj) for (int i = 0; i < s.S; ++i) obj[i] = s.obj[i];
    if (viol) for (int i = 0; i < s.S; ++i) viol[i] = s.viol[i];
    if (feasible) std::memcpy(feasible, s.feas.data(), s.S);
    if (energy) std::memcpy(energy, s.energy.data(), sizeof(double) * s.S);
    if (best_s) *best_s = s.best;
    if (step) *step = s.eval_step;
    if (best_x) QQA_CK(cudaMemcpy(best_x, r->h_descs[k].res_bestx, sizeof(uint32_t) * ((s.n + 31) / 32),
                                  cudaMemcpyDeviceToHost));
    return QQA_OK;
}

extern "C" int qqa_run_history(const qqa_run *r, int32_t k, int32_t cap, int64_t *best_obj, int32_t *at_step,
                               int32_t *count)
{
    if (!r || k < 0 || k >= r->capacity || !r->slots[k].active) return fail(QQA_EINVAL, "bad slot %d", k);
    const SlotHost &s = r->slots[k];
    const int32_t avail = std::min(s.eval_count, s.hist_cap);
    const int32_t m = std::min(avail, std::max(cap, 0));
    if (count) *count = avail;
    if (m > 0 && best_obj)
        QQA_CK(cudaMemcpy(best_obj, r->h_descs[k].hist_best, sizeof(long long) * m, cudaMemcpyDeviceToHost));
    if (m > 0 && at_step)
        QQA_CK(cudaMemcpy(at_step, r->h_descs[k].hist_step, sizeof(int32_t) * m, cudaMemcpyDeviceToHost));
    return QQA_OK;
}

extern "C" int qqa_run_slot_step(const qqa_run *r, int32_t k, int32_t *t)
{
    if (!r || k < 0 || k >= r->capacity || !r->slots[k].active) return fail(QQA_EINVAL, "bad slot %d", k);
    if (t) *t = r->slots[k].t;
    return QQA_OK;
}

extern "C" int qqa_anneal(qqa_problem *const *problems, const qqa_params *params, int32_t count,
                          const qqa_launch_config *cfg, const qqa_allocator *alloc, void *stream, qqa_run **out)
{
    qqa_run *r = nullptr;
    int rc = qqa_run_create(problems, params, count, cfg, alloc, stream, &r);
    if (rc) return rc;
    int32_t kmax = 0, re = 0;
    for (int32_t k = 0; k < count; ++k) {
        kmax = std::max(kmax, params[k].steps);
        if (params[k].round_every > 0) re = re ? std::min(re, params[k].round_every) : params[k].round_every;
    }
    int32_t done = 0;
    while (done < kmax) {
        const int32_t chunk = re > 0 ? std::min(re, kmax - done) : kmax - done;
        rc = qqa_run_steps(r, chunk, stream);
        if (!rc) {
            done += chunk;
            if (re > 0) rc = qqa_run_eval(r, stream);   // periodic rounding (the last one is the final)
        }
        if (rc) { qqa_run_destroy(r); return rc; }
    }
    if (re == 0) rc = qqa_run_eval(r, stream);
    if (!rc) rc = qqa_run_sync(r, stream);
    if (rc && rc != QQA_ENONFINITE) { qqa_run_destroy(r); return rc; }
    *out = r;
    return rc;
}

extern "C" int qqa_round_eval(qqa_run *r, void *stream, int64_t *obj, int64_t *viol, uint8_t *feasible,
                              double *energy, int32_t *best_s, uint32_t *best_x)
{
    int rc = qqa_run_eval(r, stream);
    if (rc) return rc;
    rc = qqa_run_sync(r, stream);
    if (rc && rc != QQA_ENONFINITE) return rc;
    const int rc_sync = rc;
    size_t off = 0, boff = 0;
    int32_t j = 0;
    for (int32_t k = 0; k < r->capacity; ++k) {
        const SlotHost &s = r->slots[k];
        if (!s.active) continue;
        rc = qqa_run_result(r, k, obj ? obj + off : nullptr, viol ? viol + off : nullptr,
                            feasible ? feasible + off : nullptr, energy ? energy + off : nullptr,
                            best_s ? best_s + j : nullptr, best_x ? best_x + boff : nullptr, nullptr);
        if (rc) return rc;
        off += (size_t)s.S;
        boff += (size_t)((s.n + 31) / 32);
        ++j;
    }
    return rc_sync;
}

// ------------------------------------------------------------ state / debug
static int ensure_scratch(qqa_run *r, size_t bytes, cudaStream_t st)
{
    if (r->scratch_bytes >= bytes) return QQA_OK;
    QQA_CK(cudaStreamSynchronize(st));
    r->alloc.put(r->d_scratch, st);
    r->d_scratch = (float *)r->alloc.get(bytes, st);
    r->scratch_bytes = r->d_scratch ? bytes : 0;
    if (!r->d_scratch) return fail(QQA_ENOMEM, "staging allocation of %zu bytes failed", bytes);
    return QQA_OK;
}

extern "C" int qqa_run_get_state(qqa_run *r, int32_t k, void *stream, float *X, float *m, float *v, int32_t *t)
{
    if (!r || k < 0 || k >= r->capacity || !r->slots[k].active) return fail(QQA_EINVAL, "bad slot %d", k);
    cudaStream_t st = (cudaStream_t)stream;
    const SlotHost &s = r->slots[k];
    const size_t elems = (size_t)s.n * s.S;
    int rc = ensure_scratch(r, elems * 4, st);
    if (rc) return rc;
    float *dst[3] = {X, m, v};
    for (int which = 0; which < 3; ++which) {
        if (!dst[which]) continue;
        launch_pack_state(r->d_descs, k, s.n, s.S, s.S_pad, r->prec, which, r->d_scratch, st);
        g_launches += 1;
        QQA_CK_LAUNCH("pack_state");
        QQA_CK(cudaMemcpyAsync(dst[which], r->d_scratch, elems * 4, cudaMemcpyDeviceToHost, st));
        QQA_CK(cudaStreamSynchronize(st));
    }
    if (t) *t = s.t;
    return QQA_OK;
}

extern "C" int qqa_run_set_state(qqa_run *r, int32_t k, void *stream, const float *X, const float *m, const float *v,
                                 int32_t t)
{
    if (!r || k < 0 || k >= r->capacity || !r->slots[k].active) return fail(QQA_EINVAL, "bad slot %d", k);
    if (!X || !m || !v) return fail(QQA_EINVAL, "X, m and v are required");
    SlotHost &s = r->slots[k];
    if (t < 0 || t > s.K) return fail(QQA_EINVAL, "t = %d outside [0, %d]", t, s.K);
    const size_t elems = (size_t)s.n * s.S;
    for (size_t e = 0; e < elems; ++e) {
        if (!(X[e] >= 0.0f && X[e] <= 1.0f)) return fail(QQA_EINVAL, "X[%zu] = %g outside [0, 1]", e, (double)X[e]);
        if (!(std::fabs(m[e]) <= 3.0e38f)) return fail(QQA_EINVAL, "m[%zu] = %g is not finite", e, (double)m[e]);
        if (!(v[e] >= 0.0f && v[e] <= 3.0e38f)) return fail(QQA_EINVAL, "v[%zu] = %g outside [0, inf)", e, (double)v[e]);
    }
    cudaStream_t st = (cudaStream_t)stream;
    int rc = ensure_scratch(r, elems * 12, st);
    if (rc) return rc;
    QQA_CK(cudaMemcpyAsync(r->d_scratch, X, elems * 4, cudaMemcpyHostToDevice, st));
    QQA_CK(cudaMemcpyAsync(r->d_scratch + elems, m, elems * 4, cudaMemcpyHostToDevice, st));
    QQA_CK(cudaMemcpyAsync(r->d_scratch + 2 * elems, v, elems * 4, cudaMemcpyHostToDevice, st));
    s.t = t;
    s.last_eval_t = -1;
    rc = upload_desc(r, k, st);
    if (rc) return rc;
    launch_unpack_state(r->d_descs, k, s.n, s.S, s.S_pad, r->prec, r->d_scratch, r->d_scratch + elems,
                        r->d_scratch + 2 * elems, t, st);
    g_launches += 1;
    if (r->h_descs[k].seg_cnt) QQA_CK(cudaMemsetAsync(r->h_descs[k].seg_cnt, 0, (size_t)s.prob->nlong * 4, st));
    if (s.prob->kind == QQA_MAXCLIQUE) {
        launch_colsum(r->d_descs, nullptr, 1, k, s.S_pad, r->prec, 0, 0, st);
        g_launches += 1;
    }
    if (r->dense_N) {
        launch_dense_planes(r->d_descs, k, s.n, s.S_pad, st);
        g_launches += 1;
    }
    QQA_CK_LAUNCH("set_state");
    QQA_CK(cudaStreamSynchronize(st));
    return QQA_OK;
}

extern "C" int qqa_run_step_debug(qqa_run *r, int32_t k, void *stream, float *grad)
{
    if (!r || k < 0 || k >= r->capacity || !r->slots[k].active) return fail(QQA_EINVAL, "bad slot %d", k);
    if (!grad) return fail(QQA_EINVAL, "grad is NULL");
    cudaStream_t st = (cudaStream_t)stream;
    SlotHost &s = r->slots[k];
    if (s.t >= s.K) return fail(QQA_EINVAL, "slot %d has finished its %d steps", k, s.K);
    const size_t padded = (size_t)s.n * s.S_pad, elems = (size_t)s.n * s.S;
    int rc = ensure_scratch(r, (padded + elems) * 4, st);
    if (rc) return rc;
    r->h_descs[k].grad_dbg = r->d_scratch;
    rc = upload_desc(r, k, st);
    if (rc) return rc;
    const int32_t grid = std::min(r->max_grid, r->num_tiles);
    rc = launch_step_chunk(r, 1, grid, st);
    g_launches += (unsigned long long)r->kernels_per_step + 2;
    for (auto &sl : r->slots)
        if (sl.active) sl.t = std::min(sl.t + 1, sl.K);
    r->h_descs[k].grad_dbg = nullptr;
    int rc2 = upload_desc(r, k, st);
    if (rc) return rc;
    if (rc2) return rc2;
    launch_copy_grad(r->d_descs, k, s.n, s.S, s.S_pad, r->d_scratch, r->d_scratch + padded, st);
    g_launches += 1;
    QQA_CK_LAUNCH("copy_grad");
    QQA_CK(cudaMemcpyAsync(grad, r->d_scratch + padded, elems * 4, cudaMemcpyDeviceToHost, st));
    QQA_CK(cudaStreamSynchronize(st));
    return QQA_OK;
}

extern "C" int qqa_run_debug_set_status(qqa_run *r, uint64_t nonfinite, uint64_t timeouts, void *stream)
{
    if (!r) return fail(QQA_EINVAL, "run is NULL");
    cudaStream_t st = (cudaStream_t)stream;
    const RunStatus s{(unsigned long long)nonfinite, (unsigned long long)timeouts};
    QQA_CK(cudaMemcpyAsync(r->d_status, &s, sizeof s, cudaMemcpyHostToDevice, st));
    QQA_CK(cudaStreamSynchronize(st));
    return QQA_OK;
}
