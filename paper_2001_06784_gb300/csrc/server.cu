// Query server with continuous batching (include/pivoter.h, "Serving").
//
// Three parties: callers submit queries (host CSR copied at once); a worker
// thread admits queued queries while slots and the device-memory budget
// allow, orients each admitted group in one batched launch (one block per
// graph), sizes the results from the degeneracies found, and launches the
// group's walk and combine on the next of a few streams; a completion thread
// retires groups as their events complete, frees their memory (which lets
// the worker admit more) and wakes waiters.  Orientation of a new group thus
// overlaps the walks of earlier groups, and groups on different streams
// overlap one another.
#include <algorithm>
#include <chrono>
#include <cmath>
#include <condition_variable>
#include <cstring>
#include <deque>
#include <map>
#include <memory>
#include <mutex>
#include <new>
#include <string>
#include <thread>
#include <vector>

#include "pvt_internal.cuh"

namespace pvt {
namespace {

using Clock = std::chrono::steady_clock;

enum ReqState { REQ_PENDING, REQ_RUNNING, REQ_DONE, REQ_FAILED };

constexpr size_t ALIGN = 256;
constexpr int BINOM_ROWS = BATCH_MAX_ALPHA + 3;  // every degeneracy a served graph may have
constexpr int BINOM_W = WMAX;

size_t align_up(size_t x) { return (x + ALIGN - 1) / ALIGN * ALIGN; }

// Reusable pinned host buffers (power-of-two size classes).
class PinnedPool {
public:
    ~PinnedPool()
    {
        for (auto &kv : free_)
            for (void *p : kv.second) cudaFreeHost(p);
    }
    void *get(size_t bytes, size_t *cls_out)
    {
        size_t cls = 4096;
        while (cls < bytes) cls <<= 1;
        *cls_out = cls;
        std::lock_guard<std::mutex> lk(mu_);
        auto &fl = free_[cls];
        if (!fl.empty()) {
            void *p = fl.back();
            fl.pop_back();
            return p;
        }
        void *p = nullptr;
        if (cudaMallocHost(&p, cls) != cudaSuccess) return nullptr;
        return p;
    }
    void put(void *p, size_t cls)
    {
        if (!p) return;
        std::lock_guard<std::mutex> lk(mu_);
        free_[cls].push_back(p);
    }

private:
    std::mutex mu_;
    std::map<size_t, std::vector<void *>> free_;
};

struct Request {
    uint64_t ticket = 0;
    bool direct = false;             // whole-GPU single-graph path
    int kind = 0, kmax_req = -1;
    int64_t n = 0, nnz = 0, m = 0;
    std::vector<int64_t> rp;
    std::vector<uint32_t> col;
    size_t reserve = 0;              // budget bytes held
    std::vector<void *> dallocs;     // device memory of this query
    BatchGraph desc;
    int alpha = 0, K = 0, W = 0;
    int64_t rows = 0;
    uint64_t *hres = nullptr;        // pinned result words
    size_t hres_cls = 0;
    ReqState state = REQ_PENDING;
    pvt_status status = PVT_OK;
    std::string error;
    Clock::time_point t_submit, t_done;
};
using ReqPtr = std::shared_ptr<Request>;

struct Batch {
    std::vector<ReqPtr> reqs;
    cudaStream_t stream = nullptr;
    cudaEvent_t done = nullptr;
    std::vector<void *> dallocs;
    unsigned *hctl = nullptr;        // pinned copy of the batch status word
    size_t hctl_cls = 0;
};

// Bytes a query may need on the device, from its CSR and alpha <= sqrt(2m).
size_t estimate_bytes(const Request &r, int alpha_bound)
{
    const size_t n = (size_t)r.n, m = (size_t)r.m;
    size_t b = align_up(8 * (n + 1)) + align_up(4 * (size_t)r.nnz);         // CSR
    b += 3 * align_up(4 * n) + align_up(8 * n);                             // deg, rnd, lq, tmp
    b += align_up(8 * (n + 1)) + align_up(4 * m) + align_up(4 * n);         // orow, ocol, roots
    if (r.kind == PVT_QUERY_EDGE) b += align_up(4 * m) + align_up(8 * (n + 1));
    const int W = min_words(r.n, alpha_bound);
    const size_t K = (size_t)(r.kmax_req >= 0 ? r.kmax_req + 1 : alpha_bound + 2);
    const size_t rows = r.kind == PVT_QUERY_GLOBAL ? 1 : (r.kind == PVT_QUERY_VERTEX ? n : m);
    b += align_up(rows * K * W * 8);
    if (r.kind == PVT_QUERY_GLOBAL) b += align_up((size_t)(alpha_bound + 2) * (alpha_bound + 2) * 8);
    b += align_up(8 * n);                                                   // root entries
    return b;
}

int alpha_bound(const Request &r)
{
    // degeneracy <= floor(sqrt(2m)) and <= the largest degree
    int64_t maxdeg = 0;
    for (int64_t v = 0; v < r.n; ++v) maxdeg = std::max<int64_t>(maxdeg, r.rp[v + 1] - r.rp[v]);
    const int64_t sq = (int64_t)std::floor(std::sqrt(2.0 * (double)r.m)) + 1;
    return (int)std::min<int64_t>(std::min<int64_t>(maxdeg, sq), BATCH_MAX_ALPHA);
}

}  // namespace
}  // namespace pvt

using namespace pvt;

struct pvt_server {
    pvt_server_config cfg{};
    int device = 0, num_sms = 0;
    std::mutex mu;
    std::condition_variable cv_work, cv_done, cv_complete;
    std::deque<ReqPtr> pending;
    std::deque<ReqPtr> pending_direct;  // queries for the whole-GPU path
    std::thread direct_worker;
    cudaStream_t direct_stream = nullptr;
    std::map<uint64_t, ReqPtr> all;
    std::deque<Batch *> running;
    size_t mem_used = 0;
    int inflight = 0;
    uint64_t next_ticket = 1;
    bool stop = false;
    std::thread worker, completer;
    cudaStream_t orient_stream = nullptr;
    std::vector<cudaStream_t> walk_streams;
    int next_stream = 0;
    unsigned long long *binom = nullptr;
    unsigned *binom_err = nullptr;
    PinnedPool pinned;
};

namespace pvt {
namespace {

bool can_admit(pvt_server *sv, const Request &r)
{
    return sv->inflight < sv->cfg.max_inflight && sv->mem_used + r.reserve <= sv->cfg.mem_budget;
}

void fail_request(pvt_server *sv, const ReqPtr &r, pvt_status st, const std::string &msg)
{
    for (void *p : r->dallocs) cudaFree(p);
    r->dallocs.clear();
    std::lock_guard<std::mutex> lk(sv->mu);
    r->state = REQ_FAILED;
    r->status = st;
    r->error = msg;
    r->t_done = Clock::now();
    sv->mem_used -= r->reserve;
    sv->inflight -= 1;
    sv->cv_done.notify_all();
    sv->cv_work.notify_all();
}

template <typename T>
T *carve(char *&p, size_t count)
{
    T *q = reinterpret_cast<T *>(p);
    p += align_up(sizeof(T) * std::max<size_t>(count, 1));
    return q;
}

// Orient one admitted group and launch its walk; returns after the launch.
void run_group(pvt_server *sv, std::vector<ReqPtr> &group)
{
    cudaStream_t os = sv->orient_stream;
    const int B = (int)group.size();
    auto fail_all = [&](pvt_status st, const std::string &msg) {
        for (auto &r : group) fail_request(sv, r, st, msg);
        group.clear();
    };
    // ---- 1. device memory for inputs, scratch and the DAG; copy the CSRs
    std::vector<BatchGraph> h(B);
    for (int i = 0; i < B; ++i) {
        Request &r = *group[i];
        const size_t n = (size_t)r.n, m = (size_t)r.m;
        size_t bytes = align_up(8 * (n + 1)) + align_up(4 * (size_t)std::max<int64_t>(r.nnz, 1)) +
                       3 * align_up(4 * std::max<size_t>(n, 1)) + align_up(8 * std::max<size_t>(n, 1)) +
                       align_up(8 * (n + 1)) + align_up(4 * std::max<size_t>(m, 1)) +
                       align_up(4 * std::max<size_t>(n, 1));
        if (r.kind == PVT_QUERY_EDGE) bytes += align_up(4 * std::max<size_t>(m, 1)) + align_up(8 * (n + 1));
        void *base = nullptr;
        if (cudaMallocAsync(&base, bytes, os) != cudaSuccess) { fail_all(PVT_ENOMEM, "server: device allocation failed"); return; }
        r.dallocs.push_back(base);
        char *p = static_cast<char *>(base);
        BatchGraph &G = h[i];
        G.n = r.n;
        G.nnz = r.nnz;
        int64_t *d_rp = carve<int64_t>(p, n + 1);
        uint32_t *d_col = carve<uint32_t>(p, (size_t)r.nnz);
        G.rp = d_rp;
        G.col = d_col;
        G.deg = carve<uint32_t>(p, n);
        G.rnd = carve<uint32_t>(p, n);
        G.lq = carve<uint32_t>(p, n);
        G.tmp = carve<uint32_t>(p, 2 * n);
        G.orow = carve<int64_t>(p, n + 1);
        G.ocol = carve<uint32_t>(p, m);
        G.roots = carve<uint32_t>(p, n);
        if (r.kind == PVT_QUERY_EDGE) {
            G.oeid = carve<uint32_t>(p, m);
            G.up = carve<int64_t>(p, n + 1);
        }
        G.mode = r.kind;
        cudaMemcpyAsync(d_rp, r.rp.data(), 8 * (n + 1), cudaMemcpyHostToDevice, os);
        if (r.nnz) cudaMemcpyAsync(d_col, r.col.data(), 4 * (size_t)r.nnz, cudaMemcpyHostToDevice, os);
    }
    // ---- 2. batched orientation, then the degeneracies on the host
    BatchGraph *d_graphs = nullptr;
    if (cudaMallocAsync(&d_graphs, sizeof(BatchGraph) * B, os) != cudaSuccess) { fail_all(PVT_ENOMEM, "server: descriptor allocation failed"); return; }
    cudaMemcpyAsync(d_graphs, h.data(), sizeof(BatchGraph) * B, cudaMemcpyHostToDevice, os);
    pvt_status st = batch_orient(d_graphs, B, os);
    std::vector<BatchGraph> back(B);
    cudaMemcpyAsync(back.data(), d_graphs, sizeof(BatchGraph) * B, cudaMemcpyDeviceToHost, os);
    cudaError_t ce = cudaStreamSynchronize(os);
    if (st != PVT_OK || ce != cudaSuccess) {
        cudaFree(d_graphs);
        fail_all(PVT_ECUDA, std::string("server: batched orientation failed: ") + cudaGetErrorString(ce));
        return;
    }
    // ---- 3. size every result from its degeneracy; drop failed graphs
    cudaStream_t ws = sv->walk_streams[sv->next_stream];
    sv->next_stream = (sv->next_stream + 1) % (int)sv->walk_streams.size();
    std::vector<ReqPtr> ok;
    std::vector<BatchGraph> hk;
    for (int i = 0; i < B; ++i) {
        Request &r = *group[i];
        BatchGraph G = h[i];
        std::memcpy(G.info, back[i].info, sizeof(G.info));
        if (G.info[BI_ERR]) {
            fail_request(sv, group[i], G.info[BI_ERR] == DERR_RANGE ? PVT_EINVAL : PVT_ETIMEOUT,
                         G.info[BI_ERR] == DERR_RANGE ? "server: degeneracy above 512" : "server: orientation wait timed out");
            continue;
        }
        r.alpha = (int)G.info[BI_ALPHA];
        r.W = min_words(r.n, r.alpha);
        r.K = (r.kmax_req >= 0 ? r.kmax_req : r.alpha + 1) + 1;
        r.rows = r.kind == PVT_QUERY_GLOBAL ? 1 : (r.kind == PVT_QUERY_VERTEX ? r.n : r.m);
        const size_t words = (size_t)r.rows * r.K * r.W;
        const size_t hwords = r.kind == PVT_QUERY_GLOBAL ? (size_t)(r.alpha + 2) * (r.alpha + 2) : 0;
        void *base = nullptr;
        if (cudaMallocAsync(&base, align_up(8 * std::max<size_t>(words, 1)) + align_up(8 * std::max<size_t>(hwords, 1)), ws) !=
            cudaSuccess) {
            fail_request(sv, group[i], PVT_ENOMEM, "server: result allocation failed");
            continue;
        }
        r.dallocs.push_back(base);
        char *p = static_cast<char *>(base);
        G.out = carve<unsigned long long>(p, words);
        G.hist = carve<unsigned long long>(p, hwords);
        G.hstride = r.alpha + 2;
        G.kmax = r.K - 1;
        G.W = r.W;
        cudaMemsetAsync(G.out, 0, 8 * std::max<size_t>(words, 1), ws);
        if (hwords) cudaMemsetAsync(G.hist, 0, 8 * hwords, ws);
        r.hres = static_cast<uint64_t *>(sv->pinned.get(8 * std::max<size_t>(words, 1), &r.hres_cls));
        if (!r.hres) {
            fail_request(sv, group[i], PVT_ENOMEM, "server: pinned host allocation failed");
            continue;
        }
        ok.push_back(group[i]);
        hk.push_back(G);
    }
    cudaFreeAsync(d_graphs, ws);
    const int G2 = (int)ok.size();
    if (G2 == 0) return;
    // ---- 4. root entries per (query kind, class), combine work list
    std::vector<unsigned> n_entries(3 * NCLASS, 0), off((size_t)G2 * NCLASS, 0);
    for (int g = 0; g < G2; ++g)
        for (int c = 0; c < NCLASS; ++c) {
            off[(size_t)g * NCLASS + c] = n_entries[hk[g].mode * NCLASS + c];
            n_entries[hk[g].mode * NCLASS + c] += hk[g].info[BI_CNT + c];
        }
    std::vector<int2> work;
    for (int g = 0; g < G2; ++g)
        if (hk[g].mode == BATCH_GLOBAL)
            for (int k = 0; k <= hk[g].kmax; ++k) work.push_back(make_int2(g, k));
    size_t total_entries = 0;
    for (unsigned x : n_entries) total_entries += align_up(8 * std::max<unsigned>(x, 1)) / 8;
    const size_t bbytes = align_up(sizeof(BatchGraph) * G2) + align_up(8 * total_entries) +
                          align_up(sizeof(uint64_t *) * 3 * NCLASS) + align_up(4 * off.size()) +
                          align_up(sizeof(int2) * std::max<size_t>(work.size(), 1)) + align_up(4 * 64);
    Batch *bt = new Batch();
    bt->reqs = ok;
    bt->stream = ws;
    void *bbase = nullptr;
    if (cudaMallocAsync(&bbase, bbytes, ws) != cudaSuccess) {
        for (auto &r : ok) fail_request(sv, r, PVT_ENOMEM, "server: batch allocation failed");
        delete bt;
        return;
    }
    bt->dallocs.push_back(bbase);
    char *p = static_cast<char *>(bbase);
    BatchGraph *dg = carve<BatchGraph>(p, G2);
    std::vector<uint64_t *> eptr(3 * NCLASS);
    {
        uint64_t *e = carve<uint64_t>(p, total_entries);
        for (int i = 0; i < 3 * NCLASS; ++i) {
            eptr[i] = e;
            e += align_up(8 * std::max<unsigned>(n_entries[i], 1)) / 8;
        }
    }
    uint64_t **d_eptr = carve<uint64_t *>(p, 3 * NCLASS);
    unsigned *d_off = carve<unsigned>(p, off.size());
    int2 *d_work = carve<int2>(p, std::max<size_t>(work.size(), 1));
    unsigned *d_ctl = carve<unsigned>(p, 64);
    cudaMemcpyAsync(dg, hk.data(), sizeof(BatchGraph) * G2, cudaMemcpyHostToDevice, ws);
    cudaMemcpyAsync(d_eptr, eptr.data(), sizeof(uint64_t *) * 3 * NCLASS, cudaMemcpyHostToDevice, ws);
    cudaMemcpyAsync(d_off, off.data(), 4 * off.size(), cudaMemcpyHostToDevice, ws);
    if (!work.empty()) cudaMemcpyAsync(d_work, work.data(), sizeof(int2) * work.size(), cudaMemcpyHostToDevice, ws);
    cudaMemsetAsync(d_ctl, 0, 4 * 64, ws);
    st = batch_root_entries(dg, G2, d_eptr, d_off, ws);
    if (st == PVT_OK)
        st = batch_count(dg, G2, d_work, (int)work.size(), eptr.data(), n_entries.data(), sv->binom, BINOM_W,
                         sv->num_sms, d_ctl, ws);
    // ---- 5. results to pinned host memory, completion event
    for (int g = 0; g < G2; ++g) {
        Request &r = *ok[g];
        cudaMemcpyAsync(r.hres, hk[g].out, 8 * (size_t)r.rows * r.K * r.W, cudaMemcpyDeviceToHost, ws);
    }
    bt->hctl = static_cast<unsigned *>(sv->pinned.get(4, &bt->hctl_cls));
    if (bt->hctl) cudaMemcpyAsync(bt->hctl, d_ctl, 4, cudaMemcpyDeviceToHost, ws);
    cudaEventCreateWithFlags(&bt->done, cudaEventDisableTiming);
    cudaEventRecord(bt->done, ws);
    if (st != PVT_OK || !bt->hctl) {
        cudaEventSynchronize(bt->done);
        for (auto &r : ok) fail_request(sv, r, PVT_ECUDA, "server: batched walk launch failed");
        cudaEventDestroy(bt->done);
        for (void *q : bt->dallocs) cudaFree(q);
        sv->pinned.put(bt->hctl, bt->hctl_cls);
        delete bt;
        return;
    }
    std::lock_guard<std::mutex> lk(sv->mu);
    sv->running.push_back(bt);
    sv->cv_complete.notify_all();
}

// One query through the single-graph entry points on the direct stream:
// copy the CSR, orient, count into device memory, copy the words to pinned
// host memory; the worker waits for it before the next direct query.
void run_direct(pvt_server *sv, const ReqPtr &rp)
{
    Request &r = *rp;
    cudaStream_t s = sv->direct_stream;
    const size_t n = (size_t)r.n;
    void *base = nullptr;
    if (cudaMallocAsync(&base, align_up(8 * (n + 1)) + align_up(4 * std::max<int64_t>(r.nnz, 1)), s) != cudaSuccess) {
        fail_request(sv, rp, PVT_ENOMEM, "server: device allocation failed");
        return;
    }
    r.dallocs.push_back(base);
    char *p = static_cast<char *>(base);
    int64_t *d_rp = carve<int64_t>(p, n + 1);
    uint32_t *d_col = carve<uint32_t>(p, (size_t)r.nnz);
    cudaMemcpyAsync(d_rp, r.rp.data(), 8 * (n + 1), cudaMemcpyHostToDevice, s);
    if (r.nnz) cudaMemcpyAsync(d_col, r.col.data(), 4 * (size_t)r.nnz, cudaMemcpyHostToDevice, s);
    pvt_dag *dag = nullptr;
    int32_t alpha = 0;
    pvt_status st = pvt_orient(r.n, r.nnz, d_rp, r.nnz ? d_col : nullptr, 0, s, &dag, &alpha);
    if (st != PVT_OK) {
        fail_request(sv, rp, st, "server: " + std::string(pvt_last_error()));
        return;
    }
    r.alpha = alpha;
    r.W = min_words(r.n, alpha);
    r.K = (r.kmax_req >= 0 ? r.kmax_req : alpha + 1) + 1;
    r.rows = r.kind == PVT_QUERY_GLOBAL ? 1 : (r.kind == PVT_QUERY_VERTEX ? r.n : r.m);
    const size_t words = (size_t)r.rows * r.K * r.W;
    void *out = nullptr;
    r.hres = static_cast<uint64_t *>(sv->pinned.get(8 * std::max<size_t>(words, 1), &r.hres_cls));
    if (!r.hres || cudaMallocAsync(&out, 8 * std::max<size_t>(words, 1), s) != cudaSuccess) {
        pvt_dag_free(dag);
        fail_request(sv, rp, PVT_ENOMEM, "server: result allocation failed");
        return;
    }
    r.dallocs.push_back(out);
    uint64_t *o = static_cast<uint64_t *>(out);
    st = r.kind == PVT_QUERY_GLOBAL   ? pvt_count_global(dag, r.K - 1, r.W, o, s)
         : r.kind == PVT_QUERY_VERTEX ? pvt_count_local_vertex(dag, r.K - 1, r.W, o, s)
                                      : pvt_count_local_edge(dag, r.K - 1, r.W, o, s);
    const std::string err = st == PVT_OK ? std::string() : std::string(pvt_last_error());
    if (st == PVT_OK) cudaMemcpyAsync(r.hres, o, 8 * words, cudaMemcpyDeviceToHost, s);
    const cudaError_t ce = cudaStreamSynchronize(s);
    pvt_dag_free(dag);
    if (st != PVT_OK || ce != cudaSuccess) {
        fail_request(sv, rp, st != PVT_OK ? st : PVT_ECUDA, "server: " + (st != PVT_OK ? err : cudaGetErrorString(ce)));
        return;
    }
    for (void *q : r.dallocs) cudaFreeAsync(q, s);
    std::lock_guard<std::mutex> lk(sv->mu);
    r.dallocs.clear();
    r.t_done = Clock::now();
    r.state = REQ_DONE;
    sv->mem_used -= r.reserve;
    sv->inflight -= 1;
    sv->cv_done.notify_all();
    sv->cv_work.notify_all();
}

void direct_main(pvt_server *sv)
{
    cudaSetDevice(sv->device);
    for (;;) {
        ReqPtr r;
        {
            std::unique_lock<std::mutex> lk(sv->mu);
            sv->cv_work.wait(lk, [&] {
                return sv->stop || (!sv->pending_direct.empty() && can_admit(sv, *sv->pending_direct.front()));
            });
            if (sv->pending_direct.empty() && sv->stop) break;
            if (sv->pending_direct.empty() || !can_admit(sv, *sv->pending_direct.front())) continue;
            r = sv->pending_direct.front();
            sv->pending_direct.pop_front();
            sv->mem_used += r->reserve;
            sv->inflight += 1;
            r->state = REQ_RUNNING;
        }
        run_direct(sv, r);
    }
}

void worker_main(pvt_server *sv)
{
    cudaSetDevice(sv->device);
    for (;;) {
        std::vector<ReqPtr> group;
        {
            std::unique_lock<std::mutex> lk(sv->mu);
            sv->cv_work.wait(lk, [&] { return sv->stop || (!sv->pending.empty() && can_admit(sv, *sv->pending.front())); });
            if (sv->pending.empty() && sv->stop) break;
            if (sv->pending.empty()) continue;
            while (!sv->pending.empty() && (int)group.size() < sv->cfg.max_batch && can_admit(sv, *sv->pending.front())) {
                ReqPtr r = sv->pending.front();
                sv->pending.pop_front();
                sv->mem_used += r->reserve;
                sv->inflight += 1;
                r->state = REQ_RUNNING;
                group.push_back(r);
            }
        }
        if (!group.empty()) run_group(sv, group);
    }
}

void complete_batch(pvt_server *sv, Batch *bt)
{
    const unsigned status = *bt->hctl;
    for (auto &r : bt->reqs)
        for (void *p : r->dallocs) cudaFreeAsync(p, bt->stream);
    for (void *p : bt->dallocs) cudaFreeAsync(p, bt->stream);
    std::lock_guard<std::mutex> lk(sv->mu);
    for (auto &r : bt->reqs) {
        r->dallocs.clear();
        r->t_done = Clock::now();
        if (status) {
            r->state = REQ_FAILED;
            r->status = (status & DERR_OVERFLOW) ? PVT_EOVERFLOW : PVT_EINTERNAL;
            r->error = "server: device check failed in the batched walk";
        } else {
            r->state = REQ_DONE;
        }
        sv->mem_used -= r->reserve;
        sv->inflight -= 1;
    }
    sv->pinned.put(bt->hctl, bt->hctl_cls);
    cudaEventDestroy(bt->done);
    delete bt;
    sv->cv_done.notify_all();
    sv->cv_work.notify_all();
}

void completer_main(pvt_server *sv)
{
    cudaSetDevice(sv->device);
    for (;;) {
        std::vector<Batch *> snapshot;
        {
            std::unique_lock<std::mutex> lk(sv->mu);
            sv->cv_complete.wait(lk, [&] {
                return !sv->running.empty() ||
                       (sv->stop && sv->inflight == 0 && sv->pending.empty() && sv->pending_direct.empty());
            });
            if (sv->running.empty()) break;
            snapshot.assign(sv->running.begin(), sv->running.end());
        }
        bool any = false;
        for (Batch *bt : snapshot) {
            if (cudaEventQuery(bt->done) == cudaSuccess) {
                {
                    std::lock_guard<std::mutex> lk(sv->mu);
                    sv->running.erase(std::find(sv->running.begin(), sv->running.end(), bt));
                }
                complete_batch(sv, bt);
                any = true;
            }
        }
        if (!any) std::this_thread::sleep_for(std::chrono::microseconds(20));
    }
}

}  // namespace
}  // namespace pvt

extern "C" {

pvt_status pvt_server_create(const pvt_server_config *cfg, pvt_server **out)
{
    if (!out) {
        set_error("pvt_server_create: NULL out");
        return PVT_EINVAL;
    }
    *out = nullptr;
    pvt_server *sv = new (std::nothrow) pvt_server();
    if (!sv) {
        set_error("pvt_server_create: host allocation failed");
        return PVT_ENOMEM;
    }
    if (cfg) sv->cfg = *cfg;
    if (!sv->cfg.mem_budget) sv->cfg.mem_budget = (size_t)8 << 30;
    if (sv->cfg.max_inflight <= 0) sv->cfg.max_inflight = 1024;
    if (sv->cfg.max_batch <= 0) sv->cfg.max_batch = 256;
    if (sv->cfg.streams <= 0) sv->cfg.streams = 4;
    if (sv->cfg.direct_edges == 0) sv->cfg.direct_edges = 65536;
    cudaError_t e = cudaGetDevice(&sv->device);
    if (e == cudaSuccess) e = cudaDeviceGetAttribute(&sv->num_sms, cudaDevAttrMultiProcessorCount, sv->device);
    if (e == cudaSuccess) e = cudaStreamCreateWithFlags(&sv->orient_stream, cudaStreamNonBlocking);
    if (e == cudaSuccess) e = cudaStreamCreateWithFlags(&sv->direct_stream, cudaStreamNonBlocking);
    for (int i = 0; i < sv->cfg.streams && e == cudaSuccess; ++i) {
        cudaStream_t s;
        e = cudaStreamCreateWithFlags(&s, cudaStreamNonBlocking);
        if (e == cudaSuccess) sv->walk_streams.push_back(s);
    }
    const size_t bwords = (size_t)BINOM_ROWS * (BINOM_ROWS + 1) / 2 * BINOM_W;
    if (e == cudaSuccess) e = cudaMalloc(&sv->binom, bwords * sizeof(unsigned long long));
    if (e == cudaSuccess) e = cudaMalloc(&sv->binom_err, sizeof(unsigned));
    if (e == cudaSuccess) e = cudaMemset(sv->binom_err, 0, sizeof(unsigned));
    if (e == cudaSuccess) {
        pvt_status st = build_binom(sv->binom, BINOM_ROWS, BINOM_W, sv->binom_err, sv->orient_stream);
        if (st != PVT_OK) e = cudaErrorUnknown;
    }
    if (e == cudaSuccess) e = cudaStreamSynchronize(sv->orient_stream);
    if (e != cudaSuccess) {
        pvt_status st = cuda_fail(e, "pvt_server_create");
        for (cudaStream_t s : sv->walk_streams) cudaStreamDestroy(s);
        if (sv->orient_stream) cudaStreamDestroy(sv->orient_stream);
        if (sv->direct_stream) cudaStreamDestroy(sv->direct_stream);
        cudaFree(sv->binom);
        cudaFree(sv->binom_err);
        delete sv;
        return st;
    }
    sv->worker = std::thread(worker_main, sv);
    sv->completer = std::thread(completer_main, sv);
    sv->direct_worker = std::thread(direct_main, sv);
    *out = sv;
    return PVT_OK;
}

pvt_status pvt_server_submit(pvt_server *sv, int64_t n, int64_t nnz, const int64_t *row_ptr, const uint32_t *col,
                             int32_t kind, int32_t kmax, uint64_t *ticket)
{
    if (!sv || !ticket || n < 0 || n > 0xFFFFFFFEll || nnz < 0 || (nnz & 1) || !row_ptr || (nnz > 0 && !col) ||
        kind < PVT_QUERY_GLOBAL || kind > PVT_QUERY_EDGE || (row_ptr[n] != nnz)) {
        set_error("pvt_server_submit: invalid argument");
        return PVT_EINVAL;
    }
    auto r = std::make_shared<Request>();
    r->kind = kind;
    r->kmax_req = kmax < 0 ? -1 : kmax;
    r->n = n;
    r->nnz = nnz;
    r->m = nnz / 2;
    r->rp.assign(row_ptr, row_ptr + n + 1);
    r->col.assign(col, col + nnz);
    r->direct = sv->cfg.direct_edges > 0 && r->m >= sv->cfg.direct_edges;
    const int ab = alpha_bound(*r);
    // the direct path's dag also holds its own scratch (frame buffer, queues)
    r->reserve = estimate_bytes(*r, ab) + (r->direct ? ((size_t)256 << 20) : 0);
    if (r->reserve > sv->cfg.mem_budget) {
        set_error("pvt_server_submit: query needs more device memory than the server's budget");
        return PVT_ENOMEM;
    }
    r->t_submit = Clock::now();
    {
        std::lock_guard<std::mutex> lk(sv->mu);
        if (sv->stop) {
            set_error("pvt_server_submit: server is stopping");
            return PVT_EINVAL;
        }
        r->ticket = sv->next_ticket++;
        sv->all[r->ticket] = r;
        (r->direct ? sv->pending_direct : sv->pending).push_back(r);
    }
    sv->cv_work.notify_all();
    *ticket = r->ticket;
    return PVT_OK;
}

pvt_status pvt_server_wait(pvt_server *sv, uint64_t ticket, int32_t timeout_ms, int32_t *done)
{
    if (!sv || !done) {
        set_error("pvt_server_wait: invalid argument");
        return PVT_EINVAL;
    }
    std::unique_lock<std::mutex> lk(sv->mu);
    auto it = sv->all.find(ticket);
    if (it == sv->all.end()) {
        set_error("pvt_server_wait: unknown ticket");
        return PVT_EINVAL;
    }
    ReqPtr r = it->second;
    auto ready = [&] { return r->state == REQ_DONE || r->state == REQ_FAILED; };
    if (timeout_ms < 0) sv->cv_done.wait(lk, ready);
    else sv->cv_done.wait_for(lk, std::chrono::milliseconds(timeout_ms), ready);
    *done = ready() ? 1 : 0;
    return PVT_OK;
}

pvt_status pvt_server_result(pvt_server *sv, uint64_t ticket, int64_t *rows, int32_t *K, int32_t *W, uint64_t *out,
                             size_t out_words, double *latency_s)
{
    if (!sv) {
        set_error("pvt_server_result: NULL server");
        return PVT_EINVAL;
    }
    ReqPtr r;
    {
        std::lock_guard<std::mutex> lk(sv->mu);
        auto it = sv->all.find(ticket);
        if (it == sv->all.end()) {
            set_error("pvt_server_result: unknown ticket");
            return PVT_EINVAL;
        }
        r = it->second;
        if (r->state == REQ_FAILED) {
            set_error(r->error);
            pvt_status st = r->status;
            if (out) {
                sv->all.erase(it);
                sv->pinned.put(r->hres, r->hres_cls);
                r->hres = nullptr;
            }
            return st;
        }
        if (r->state != REQ_DONE) {
            set_error("pvt_server_result: query not finished");
            return PVT_EINVAL;
        }
    }
    if (rows) *rows = r->rows;
    if (K) *K = r->K;
    if (W) *W = r->W;
    if (!out) return PVT_OK;
    const size_t words = (size_t)r->rows * r->K * r->W;
    if (out_words < words) {
        set_error("pvt_server_result: output buffer too small");
        return PVT_EINVAL;
    }
    std::memcpy(out, r->hres, 8 * words);
    if (latency_s) *latency_s = std::chrono::duration<double>(r->t_done - r->t_submit).count();
    std::lock_guard<std::mutex> lk(sv->mu);
    sv->pinned.put(r->hres, r->hres_cls);
    r->hres = nullptr;
    sv->all.erase(ticket);
    return PVT_OK;
}

void pvt_server_destroy(pvt_server *sv)
{
    if (!sv) return;
    {
        std::lock_guard<std::mutex> lk(sv->mu);
        sv->stop = true;
    }
    sv->cv_work.notify_all();
    if (sv->worker.joinable()) sv->worker.join();
    if (sv->direct_worker.joinable()) sv->direct_worker.join();
    {
        std::lock_guard<std::mutex> lk(sv->mu);
        sv->cv_complete.notify_all();
    }
    if (sv->completer.joinable()) sv->completer.join();
    cudaDeviceSynchronize();
    for (auto &kv : sv->all)
        if (kv.second->hres) sv->pinned.put(kv.second->hres, kv.second->hres_cls);
    for (cudaStream_t s : sv->walk_streams) cudaStreamDestroy(s);
    cudaStreamDestroy(sv->orient_stream);
    cudaStreamDestroy(sv->direct_stream);
    cudaFree(sv->binom);
    cudaFree(sv->binom_err);
    delete sv;
}

}  // extern "C"
