// server.cu -- continuous-batching solve server on top of the run API.
//
// Requests (one graph plus its hyper-parameters) arrive at any time and wait
// in a queue. At each pump the server
//   1. admits queued requests in arrival order, with backfill (see admit), while
//      the HBM budget - every request is charged the exact device bytes its
//      graph and state take - and a free slot of its replica class allow (graph
//      upload, state allocation and initial draw happen here),
//   2. advances every class run by one or more chunks of steps (a class with
//      less work per step runs more chunks in the time the largest class
//      takes for one), each class on its own stream so the classes' work
//      overlaps on the device; inside a class the requests share each step
//      launch (one tile list),
//   3. evaluates (projection rounding and exact costs) and retires the
//      requests that reached their own step count, freeing slot and memory.
// A request therefore joins or leaves a batch between chunks of steps, not
// only when the whole batch is done.
//
// Replica classes: S is rounded up to a power of two (at least 8) and each
// class run has one fixed launch shape, so a request's trajectory does not
// depend on which other requests share its launches.
#include <algorithm>
#include <chrono>
#include <cstring>
#include <deque>
#include <map>
#include <memory>
#include <new>
#include <string>
#include <vector>

#include "../../include/qqa.h"

namespace qqa {
int64_t request_device_bytes(int32_t kind, int32_t n, const int32_t *row_ptr, bool weighted, const qqa_params *prm);
}

namespace {

double now_s()
{
    using namespace std::chrono;
    return duration<double>(steady_clock::now().time_since_epoch()).count();
}

struct Request {
    int64_t id = 0;
    int32_t kind = 0, n = 0;
    std::vector<int32_t> row_ptr, col, w;
    qqa_params prm{};
    int32_t state = QQA_REQ_QUEUED;
    int32_t error = QQA_OK;
    int64_t bytes = 0;
    int32_t cls = -1, slot = -1;
    int32_t passed_over = 0;          // pumps in which later requests were admitted before it
    qqa_problem *prob = nullptr;
    double t_submit = 0, t_admit = 0, t_done = 0;
    // results (filled at retirement)
    std::vector<int64_t> obj, viol;
    std::vector<uint8_t> feas;
    std::vector<double> energy;
    std::vector<uint32_t> best_x;
    std::vector<int64_t> hist;
    int32_t best_s = -1;
};

struct ClassRun {
    int32_t S_class = 0;
    qqa_run *run = nullptr;
    cudaStream_t stream = nullptr;
    std::vector<int64_t> slot_req;   // request id per slot (-1 free)
};

}  // namespace

struct qqa_server {
    int64_t budget = 0, used = 0;
    int32_t chunk = 50, slots_per_class = 64, precision = QQA_FP32;
    qqa_launch_config cfg{};
    bool has_cfg = false;
    qqa_allocator alloc{};
    bool has_alloc = false;
    int64_t next_id = 1;
    std::deque<int64_t> queue;
    std::map<int64_t, std::unique_ptr<Request>> reqs;
    std::map<int32_t, ClassRun> classes;
    std::string err;
};

static int32_t class_of(int32_t S)
{
    int32_t c = 8;
    while (c < S) c <<= 1;
    return c;
}

extern "C" int64_t qqa_request_bytes(int32_t n, int64_t nnz, int32_t S, int32_t precision, int32_t weighted)
{
    const int64_t vec = precision == QQA_FP32 ? 4 : 8;
    const int64_t S_pad = (S + vec - 1) / vec * vec;
    const int64_t elems = (int64_t)n * S_pad;
    const int64_t state = precision == QQA_FP32 ? elems * 16 : elems * 12;   // X x2, (master), m, v
    const int64_t evalb = (int64_t)n * ((S + 31) / 32) * 4 + S_pad * 56 + ((n + 31) / 32) * 4 + 4096;
    const int64_t graph = 4 * ((int64_t)n + 1) + 4 * nnz * (weighted ? 2 : 1);
    return state + evalb + graph;
}

// Bytes a class run holds whatever its requests: descriptors, status, tile
// counters and the smallest work lists.
static int64_t class_fixed_bytes(int32_t slots) { return (int64_t)slots * 512 + 8192; }

extern "C" int qqa_server_create(int64_t hbm_budget_bytes, int32_t chunk_steps, int32_t slots_per_class,
                                 int32_t precision, const qqa_launch_config *cfg, const qqa_allocator *alloc,
                                 qqa_server **out)
{
    if (!out || hbm_budget_bytes <= 0 || chunk_steps < 1 || chunk_steps > 50 || slots_per_class < 1 ||
        (precision != QQA_FP32 && precision != QQA_BF16))
        return QQA_EINVAL;
    qqa_server *s = new (std::nothrow) qqa_server();
    if (!s) return QQA_ENOMEM;
    s->budget = hbm_budget_bytes;
    s->chunk = chunk_steps;
    s->slots_per_class = slots_per_class;
    s->precision = precision;
    if (cfg) { s->cfg = *cfg; s->has_cfg = true; }
    if (alloc && alloc->alloc && alloc->free) { s->alloc = *alloc; s->has_alloc = true; }
    *out = s;
    return QQA_OK;
}

extern "C" int qqa_server_submit(qqa_server *s, int32_t kind, int32_t n, const int32_t *row_ptr, const int32_t *col,
                                 const int32_t *w, const qqa_params *prm, int64_t *request_id)
{
    if (!s || !row_ptr || !prm || n < 1 || !request_id) return QQA_EINVAL;
    if (prm->precision != s->precision || prm->S < 1 || prm->S > 1024) return QQA_EINVAL;
    const int64_t nnz = row_ptr[n];
    auto r = std::unique_ptr<Request>(new (std::nothrow) Request());
    if (!r) return QQA_ENOMEM;
    r->id = s->next_id++;
    r->kind = kind;
    r->n = n;
    r->row_ptr.assign(row_ptr, row_ptr + n + 1);
    if (nnz > 0) r->col.assign(col, col + nnz);
    if (w && nnz > 0) r->w.assign(w, w + nnz);
    r->prm = *prm;
    r->bytes = qqa::request_device_bytes(kind, n, row_ptr, w != nullptr, prm);
    r->t_submit = now_s();
    if (r->bytes > s->budget) {   // can never fit: rejected now
        r->state = QQA_REQ_FAILED;
        r->error = QQA_ENOMEM;
        r->t_done = r->t_submit;
    } else {
        s->queue.push_back(r->id);
    }
    *request_id = r->id;
    s->reqs[r->id] = std::move(r);
    return QQA_OK;
}

static ClassRun *get_class(qqa_server *s, int32_t cls, int *rc)
{
    auto it = s->classes.find(cls);
    if (it != s->classes.end()) return &it->second;
    ClassRun c;
    c.S_class = cls;
    if (cudaStreamCreateWithFlags(&c.stream, cudaStreamNonBlocking) != cudaSuccess) {
        (void)cudaGetLastError();
        *rc = QQA_ECUDA;
        return nullptr;
    }
    *rc = qqa_run_create_empty(s->slots_per_class, cls, s->precision, s->has_cfg ? &s->cfg : nullptr,
                               s->has_alloc ? &s->alloc : nullptr, c.stream, &c.run);
    if (*rc) {
        cudaStreamDestroy(c.stream);
        return nullptr;
    }
    c.slot_req.assign(s->slots_per_class, -1);
    s->used += class_fixed_bytes(s->slots_per_class);
    auto res = s->classes.emplace(cls, c);
    return &res.first->second;
}

static void release(qqa_server *s, Request *r)
{
    if (r->cls >= 0 && r->slot >= 0) {
        ClassRun &c = s->classes[r->cls];
        qqa_run_remove(c.run, r->slot, c.stream);
        c.slot_req[r->slot] = -1;
    }
    if (r->prob) qqa_destroy_problem(r->prob);
    r->prob = nullptr;
    r->slot = -1;
    s->used -= r->bytes;
}

// Pumps a request that does not fit the budget may be passed over by later,
// smaller ones before admission waits for it.
static const int32_t kMaxPassOver = 32;

// Admission: arrival order with backfill. A request that does not fit the HBM
// budget now is passed over and later requests that do fit are admitted
// (small requests do not queue behind a large one); after kMaxPassOver such
// pumps nothing more is admitted ahead of it, so it cannot wait forever. A
// request whose replica class has no free slot waits without holding up the
// other classes.
static void admit(qqa_server *s)
{
    for (auto it = s->queue.begin(); it != s->queue.end();) {
        Request *r = s->reqs[*it].get();
        const int32_t cls = class_of(r->prm.S);
        const bool has_class = s->classes.count(cls) != 0;
        const int64_t need = r->bytes + (has_class ? 0 : class_fixed_bytes(s->slots_per_class));
        if (s->used + need > s->budget) {
            if (++r->passed_over >= kMaxPassOver) break;   // it goes first from now on
            ++it;
            continue;
        }
        int rc = QQA_OK;
        ClassRun *c = get_class(s, cls, &rc);
        if (!c) {
            r->state = QQA_REQ_FAILED;
            r->error = rc;
            r->t_done = now_s();
            it = s->queue.erase(it);
            continue;
        }
        if (std::find(c->slot_req.begin(), c->slot_req.end(), -1) == c->slot_req.end()) {   // class full
            ++it;
            continue;
        }
        it = s->queue.erase(it);
        s->used += r->bytes;
        rc = qqa_create_problem(r->kind, r->n, r->row_ptr.data(), r->col.empty() ? nullptr : r->col.data(),
                                r->w.empty() ? nullptr : r->w.data(), s->has_alloc ? &s->alloc : nullptr,
                                c->stream, &r->prob);
        int32_t slot = -1;
        if (!rc) rc = qqa_run_add(c->run, r->prob, &r->prm, c->stream, &slot);
        if (rc) {   // e.g. an allocation failed: this request fails, the others go on
            r->state = QQA_REQ_FAILED;
            r->error = rc;
            r->t_done = now_s();
            release(s, r);
            continue;
        }
        r->cls = cls;
        r->slot = slot;
        c->slot_req[slot] = r->id;
        r->state = QQA_REQ_RUNNING;
        r->t_admit = now_s();
        std::vector<int32_t>().swap(r->col);   // the device copy is what matters now
        std::vector<int32_t>().swap(r->w);
    }
}

// Work of one step of a class: the state elements of its running requests.
static double class_work(const qqa_server *s, const ClassRun &c)
{
    double w = 0.0;
    for (int64_t id : c.slot_req)
        if (id >= 0) {
            const Request *r = s->reqs.at(id).get();
            w += (double)r->n * (double)c.S_class;
        }
    return w;
}

extern "C" int qqa_server_pump(qqa_server *s, int32_t *n_running, int32_t *n_queued, int32_t *n_finished)
{
    if (!s) return QQA_EINVAL;
    admit(s);
    // Every class with running requests advances on its own stream, so the
    // classes run side by side; a pump lasts about as long as the class with
    // the most work per step needs for one chunk, and a class with k times less
    // work runs up to k chunks (at most 8) in that time, so small requests are
    // not held to the pace of large ones.
    double max_work = 0.0;
    for (auto &kv : s->classes) max_work = std::max(max_work, class_work(s, kv.second));
    for (auto &kv : s->classes) {
        ClassRun &c = kv.second;
        const double w = class_work(s, c);
        if (w <= 0.0) continue;
        const int32_t chunks = (int32_t)std::max(1.0, std::min(8.0, std::floor(max_work / w)));
        for (int32_t k = 0; k < chunks; ++k) {   // a rounding after every chunk: the same history in any mix
            int rc = qqa_run_steps(c.run, s->chunk, c.stream);
            if (!rc) rc = qqa_run_eval(c.run, c.stream);
            if (rc) return rc;
        }
    }
    int32_t finished = 0;
    for (auto &kv : s->classes) {
        ClassRun &c = kv.second;
        bool any = false;
        for (int64_t id : c.slot_req) any |= id >= 0;
        if (!any) continue;
        const int rc = qqa_run_sync(c.run, c.stream);
        const bool nonfinite = rc == QQA_ENONFINITE;
        if (rc && !nonfinite) return rc;
        for (int32_t k = 0; k < (int32_t)c.slot_req.size(); ++k) {
            if (c.slot_req[k] < 0) continue;
            Request *r = s->reqs[c.slot_req[k]].get();
            int32_t t = 0;
            qqa_run_slot_step(c.run, k, &t);
            if (t < r->prm.steps) continue;
            const int32_t S = r->prm.S;
            r->obj.resize(S);
            r->viol.resize(S);
            r->feas.resize(S);
            r->energy.resize(S);
            r->best_x.resize((r->n + 31) / 32);
            qqa_run_result(c.run, k, r->obj.data(), r->viol.data(), r->feas.data(), r->energy.data(), &r->best_s,
                           r->best_x.data(), nullptr);
            int32_t cnt = 0;
            qqa_run_history(c.run, k, 0, nullptr, nullptr, &cnt);
            r->hist.resize(cnt);
            std::vector<int32_t> at(cnt);
            if (cnt) qqa_run_history(c.run, k, cnt, r->hist.data(), at.data(), &cnt);
            r->state = nonfinite ? QQA_REQ_FAILED : QQA_REQ_DONE;
            r->error = nonfinite ? QQA_ENONFINITE : QQA_OK;
            r->t_done = now_s();
            release(s, r);
            ++finished;
        }
    }
    if (n_running || n_queued) {
        int32_t running = 0;
        for (auto &kv : s->classes)
            for (int64_t id : kv.second.slot_req) running += id >= 0;
        if (n_running) *n_running = running;
        if (n_queued) *n_queued = (int32_t)s->queue.size();
    }
    if (n_finished) *n_finished = finished;
    return QQA_OK;
}

extern "C" int qqa_server_cancel(qqa_server *s, int64_t id)
{
    if (!s) return QQA_EINVAL;
    auto it = s->reqs.find(id);
    if (it == s->reqs.end()) return QQA_EINVAL;
    Request *r = it->second.get();
    if (r->state == QQA_REQ_QUEUED) {
        s->queue.erase(std::remove(s->queue.begin(), s->queue.end(), id), s->queue.end());
    } else if (r->state == QQA_REQ_RUNNING) {
        ClassRun &c = s->classes[r->cls];
        cudaStreamSynchronize(c.stream);
        release(s, r);
    } else {
        return QQA_OK;
    }
    r->state = QQA_REQ_CANCELLED;
    r->t_done = now_s();
    return QQA_OK;
}

extern "C" int qqa_server_poll(const qqa_server *s, int64_t id, qqa_request_info *info)
{
    if (!s || !info) return QQA_EINVAL;
    auto it = s->reqs.find(id);
    if (it == s->reqs.end()) return QQA_EINVAL;
    const Request *r = it->second.get();
    info->state = r->state;
    info->error = r->error;
    info->S = r->prm.S;
    info->n = r->n;
    info->best_s = r->best_s;
    info->best_obj = (r->state == QQA_REQ_DONE && r->best_s >= 0) ? r->obj[r->best_s] : INT64_MIN;
    info->feasible = 0;
    for (uint8_t f : r->feas) info->feasible += f;
    info->t_submit = r->t_submit;
    info->t_admit = r->t_admit;
    info->t_done = r->t_done;
    info->bytes = r->bytes;
    info->evaluations = (int32_t)r->hist.size();
    return QQA_OK;
}

extern "C" int qqa_server_result(const qqa_server *s, int64_t id, int64_t *obj, int64_t *viol, uint8_t *feasible,
                                 double *energy, uint32_t *best_x, int64_t *history)
{
    if (!s) return QQA_EINVAL;
    auto it = s->reqs.find(id);
    if (it == s->reqs.end() || it->second->state != QQA_REQ_DONE) return QQA_EBUSY;
    const Request *r = it->second.get();
    const size_t S = r->obj.size();
    if (obj) std::memcpy(obj, r->obj.data(), S * 8);
    if (viol) std::memcpy(viol, r->viol.data(), S * 8);
    if (feasible) std::memcpy(feasible, r->feas.data(), S);
    if (energy) std::memcpy(energy, r->energy.data(), S * 8);
    if (best_x) std::memcpy(best_x, r->best_x.data(), r->best_x.size() * 4);
    if (history) std::memcpy(history, r->hist.data(), r->hist.size() * 8);
    return QQA_OK;
}

extern "C" int qqa_server_stats(const qqa_server *s, int64_t *used_bytes, int32_t *classes)
{
    if (!s) return QQA_EINVAL;
    if (used_bytes) *used_bytes = s->used;
    if (classes) *classes = (int32_t)s->classes.size();
    return QQA_OK;
}

extern "C" void qqa_server_destroy(qqa_server *s)
{
    if (!s) return;
    for (auto &kv : s->reqs)
        if (kv.second->state == QQA_REQ_RUNNING) release(s, kv.second.get());
    for (auto &kv : s->classes) {
        if (kv.second.run) qqa_run_destroy(kv.second.run);
        if (kv.second.stream) cudaStreamDestroy(kv.second.stream);
    }
    delete s;
}
