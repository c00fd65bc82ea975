// C ABI entry points of libpivoter (declared in include/pivoter.h).
#include <mutex>
#include <new>
#include <vector>
#include <string>

#include "pvt_internal.cuh"

namespace pvt {

static thread_local std::string t_error;

void set_error(const std::string &msg) { t_error = msg; }

pvt_status cuda_fail(cudaError_t e, const char *what)
{
    set_error(std::string(what) + ": " + cudaGetErrorString(e));
    return e == cudaErrorMemoryAllocation ? PVT_ENOMEM : PVT_ECUDA;
}

int32_t min_words(int64_t n, int32_t alpha)
{
    int bits = 0;
    for (uint64_t x = (uint64_t)n; x; x >>= 1) ++bits;
    int w = (bits + alpha + 1 + 63) / 64;
    return w < 1 ? 1 : w;
}

pvt_status check_device(pvt_dag *g, cudaStream_t s, const char *what)
{
    PVT_CK(cudaMemcpyAsync(g->h_err, g->d_err, sizeof(unsigned), cudaMemcpyDeviceToHost, s));
    PVT_CK(cudaStreamSynchronize(s));
    unsigned e = *g->h_err;
    if (!e) return PVT_OK;
    std::string w(what);
    if (e & DERR_NOTSIMPLE) { set_error(w + ": CSR is not a simple undirected graph"); return PVT_ENOTSIMPLE; }
    if (e & DERR_TIMEOUT) { set_error(w + ": device-side wait timed out"); return PVT_ETIMEOUT; }
    if (e & DERR_OVERFLOW) { set_error(w + ": multi-word overflow"); return PVT_EOVERFLOW; }
    if (e & DERR_STACK) { set_error(w + ": DFS stack capacity exceeded"); return PVT_EINTERNAL; }
    if (e & DERR_CHECK) { set_error(w + ": internal consistency check of the root paths failed"); return PVT_EINTERNAL; }
    set_error(w + ": device index check failed");
    return PVT_EINTERNAL;
}

void phase_begin(pvt_dag *g, int ph, cudaStream_t s)
{
    if (!g->profiling || g->capturing) return;
    cudaEventRecord(g->ev_t0[ph], s);
    g->phase_used[ph] = true;
}

void phase_end(pvt_dag *g, int ph, cudaStream_t s)
{
    if (g->profiling && !g->capturing) cudaEventRecord(g->ev_t1[ph], s);
}

void stats_reset(pvt_dag *g)
{
    g->stats = pvt_stats{};
    for (int i = 0; i < NPHASE; ++i) g->phase_used[i] = false;
}

// Per-device resources that every dag needs whatever its graph -- status
// and statistics words, pinned host copies, queue counters, side streams,
// events, the Pascal table -- outlive their dag: pvt_dag_free hands them
// back to a pool and the next pvt_orient on that device takes them, which
// saves their creation (synchronous allocations, stream and event set-up)
// on every call.
struct DagRes {
    int device = -1;
    unsigned *d_err = nullptr, *d_q = nullptr, *h_err = nullptr;
    unsigned long long *d_stats = nullptr, *h_stats = nullptr;
    uint32_t *qctl = nullptr;
    cudaEvent_t ev_t0[NPHASE] = {}, ev_t1[NPHASE] = {}, ev_fork = nullptr, ev_join[NCLASS] = {};
    cudaStream_t side[NCLASS] = {};
    DevBuf<unsigned long long> binom;
    int binom_rows = 0, binom_W = 0;
};

static std::mutex g_res_mu;
static std::vector<DagRes> g_res_pool;

static cudaError_t res_create(int device, DagRes &r)
{
    r.device = device;
    cudaError_t e = cudaMalloc(&r.d_err, sizeof(unsigned));
    if (e == cudaSuccess) e = cudaMalloc(&r.d_q, 16 * sizeof(unsigned));
    if (e == cudaSuccess) e = cudaMalloc(&r.d_stats, 16 * sizeof(unsigned long long));
    if (e == cudaSuccess) e = cudaMalloc(&r.qctl, NCLASS * 128 * sizeof(uint32_t));
    for (int i = 0; i < NPHASE && e == cudaSuccess; ++i) {
        e = cudaEventCreate(&r.ev_t0[i]);
        if (e == cudaSuccess) e = cudaEventCreate(&r.ev_t1[i]);
    }
    if (e == cudaSuccess) e = cudaMallocHost(&r.h_err, sizeof(unsigned));
    if (e == cudaSuccess) e = cudaMallocHost(&r.h_stats, 16 * sizeof(unsigned long long));
    if (e == cudaSuccess) e = cudaEventCreateWithFlags(&r.ev_fork, cudaEventDisableTiming);
    for (int c = 0; c < NCLASS && e == cudaSuccess; ++c) {
        e = cudaStreamCreateWithFlags(&r.side[c], cudaStreamNonBlocking);
        if (e == cudaSuccess) e = cudaEventCreateWithFlags(&r.ev_join[c], cudaEventDisableTiming);
    }
    return e;
}

static void res_destroy(DagRes &r)
{
    for (int c = 0; c < NCLASS; ++c) {
        if (r.side[c]) { cudaStreamSynchronize(r.side[c]); cudaStreamDestroy(r.side[c]); }
        if (r.ev_join[c]) cudaEventDestroy(r.ev_join[c]);
    }
    if (r.ev_fork) cudaEventDestroy(r.ev_fork);
    for (int i = 0; i < NPHASE; ++i) {
        if (r.ev_t0[i]) cudaEventDestroy(r.ev_t0[i]);
        if (r.ev_t1[i]) cudaEventDestroy(r.ev_t1[i]);
    }
    cudaFree(r.d_err);
    cudaFree(r.d_q);
    cudaFree(r.d_stats);
    cudaFree(r.qctl);
    cudaFree(r.binom.p);
    if (r.h_err) cudaFreeHost(r.h_err);
    if (r.h_stats) cudaFreeHost(r.h_stats);
    r = DagRes{};
}

// A resource set for `device` (current), from the pool or new.
static cudaError_t res_take(int device, DagRes &r)
{
    {
        std::lock_guard<std::mutex> lk(g_res_mu);
        for (size_t i = 0; i < g_res_pool.size(); ++i)
            if (g_res_pool[i].device == device) {
                r = g_res_pool[i];
                g_res_pool[i] = g_res_pool.back();
                g_res_pool.pop_back();
                return cudaSuccess;
            }
    }
    cudaError_t e = res_create(device, r);
    if (e != cudaSuccess) res_destroy(r);
    return e;
}

static void res_to_dag(const DagRes &r, pvt_dag *g)
{
    g->d_err = r.d_err;
    g->d_q = r.d_q;
    g->d_stats = r.d_stats;
    g->qctl = r.qctl;
    g->h_err = r.h_err;
    g->h_stats = r.h_stats;
    for (int i = 0; i < NPHASE; ++i) {
        g->ev_t0[i] = r.ev_t0[i];
        g->ev_t1[i] = r.ev_t1[i];
    }
    g->ev_fork = r.ev_fork;
    for (int c = 0; c < NCLASS; ++c) {
        g->ev_join[c] = r.ev_join[c];
        g->side[c] = r.side[c];
    }
    g->binom = r.binom;
    g->binom_rows = r.binom_rows;
    g->binom_W = r.binom_W;
}

static void dag_release(pvt_dag *g)
{
    if (!g) return;
    drop_graph(g);
    // nothing of this dag is in flight once its side streams are idle: every
    // entry point synchronises the caller's stream before it returns
    for (int c = 0; c < NCLASS; ++c)
        if (g->side[c]) cudaStreamSynchronize(g->side[c]);
    cudaStream_t fs = g->side[0];
    auto release = [&](void *p) {
        if (p) cudaFreeAsync(p, fs);
    };
    release(g->rnd);
    release(g->core);
    release(g->orow);
    release(g->ocol);
    release(g->oeid);
    release(g->roots);
    release(g->hist.p);
    for (int c = 0; c < NCLASS; ++c) {
        release(g->rootbuf[c].p);
        release(g->qframes[c].p);
        release(g->qready[c].p);
        release(g->gstack[c].p);
        release(g->etab[c].p);
    }
    release(g->cframes.p);
    release(g->range_roots.p);
    release(g->range_pos.p);
    if (fs) cudaStreamSynchronize(fs);
    DagRes r;
    r.device = g->device;
    r.d_err = g->d_err;
    r.d_q = g->d_q;
    r.d_stats = g->d_stats;
    r.qctl = g->qctl;
    r.h_err = g->h_err;
    r.h_stats = g->h_stats;
    for (int i = 0; i < NPHASE; ++i) {
        r.ev_t0[i] = g->ev_t0[i];
        r.ev_t1[i] = g->ev_t1[i];
    }
    r.ev_fork = g->ev_fork;
    for (int c = 0; c < NCLASS; ++c) {
        r.ev_join[c] = g->ev_join[c];
        r.side[c] = g->side[c];
    }
    r.binom = g->binom;
    r.binom_rows = g->binom_rows;
    r.binom_W = g->binom_W;
    if (r.d_err && r.side[NCLASS - 1] && r.h_stats) {
        std::lock_guard<std::mutex> lk(g_res_mu);
        g_res_pool.push_back(r);
    } else {
        res_destroy(r);  // a set that was never complete
    }
    delete g;
}

}  // namespace pvt

using namespace pvt;

extern "C" {

pvt_status pvt_orient(int64_t n, int64_t nnz, const int64_t *row_ptr, const uint32_t *col,
                      uint32_t flags, void *stream, pvt_dag **dag_out, int32_t *alpha_out)
{
    const HostRange range("pvt_orient");
    if (!dag_out || n < 0 || n > 0xFFFFFFFEll || nnz < 0 || (nnz & 1) || (n > 0 && !row_ptr) ||
        (nnz > 0 && !col) || (flags & ~(PVT_VALIDATE | PVT_PROFILE))) {
        set_error("pvt_orient: invalid argument");
        return PVT_EINVAL;
    }
    *dag_out = nullptr;
    cudaStream_t s = (cudaStream_t)stream;
    pvt_dag *g = new (std::nothrow) pvt_dag();
    if (!g) {
        set_error("pvt_orient: host allocation failed");
        return PVT_ENOMEM;
    }
    pvt_status st = PVT_OK;
    auto fail = [&](pvt_status x) { dag_release(g); return x; };
    cudaError_t e = cudaGetDevice(&g->device);
    if (e == cudaSuccess) e = cudaDeviceGetAttribute(&g->num_sms, cudaDevAttrMultiProcessorCount, g->device);
    if (e == cudaSuccess) {
        DagRes r;
        e = res_take(g->device, r);
        if (e == cudaSuccess) res_to_dag(r, g);
    }
    if (e == cudaSuccess) {
        // keep stream-ordered scratch cached across calls instead of handing it
        // back to the driver at every synchronisation (process-wide setting)
        cudaMemPool_t pool;
        e = cudaDeviceGetDefaultMemPool(&pool, g->device);
        uint64_t keep = ~0ull;
        if (e == cudaSuccess) e = cudaMemPoolSetAttribute(pool, cudaMemPoolAttrReleaseThreshold, &keep);
    }
    if (e != cudaSuccess) return fail(cuda_fail(e, "pvt_orient: setup"));
    g->n = n;
    g->nnz = nnz;
    g->m = nnz / 2;
    g->row_ptr = row_ptr;
    g->col = col;
    g->profiling = (flags & PVT_PROFILE) != 0;
    stats_reset(g);
    st = orient_build(g, flags, s);
    if (st != PVT_OK) return fail(st);
    if (alpha_out) *alpha_out = g->alpha;
    *dag_out = g;
    return PVT_OK;
}

pvt_status pvt_dag_info(const pvt_dag *dag, int64_t *n, int64_t *m, int32_t *alpha, int32_t *min_w)
{
    if (!dag) {
        set_error("pvt_dag_info: NULL dag");
        return PVT_EINVAL;
    }
    if (n) *n = dag->n;
    if (m) *m = dag->m;
    if (alpha) *alpha = dag->alpha;
    if (min_w) *min_w = min_words(dag->n, dag->alpha);
    return PVT_OK;
}

pvt_status pvt_dag_cores(const pvt_dag *dag, uint32_t *core, void *stream)
{
    if (!dag || (!core && dag->n > 0)) {
        set_error("pvt_dag_cores: invalid argument");
        return PVT_EINVAL;
    }
    if (dag->n > 0)
        PVT_CK(cudaMemcpyAsync(core, dag->core, (size_t)dag->n * sizeof(uint32_t), cudaMemcpyDeviceToDevice,
                               (cudaStream_t)stream));
    return PVT_OK;
}

pvt_status pvt_dag_out_lists(const pvt_dag *dag, int64_t *orow, uint32_t *ocol, void *stream)
{
    if (!dag || !orow || (!ocol && dag->m > 0)) {
        set_error("pvt_dag_out_lists: invalid argument");
        return PVT_EINVAL;
    }
    cudaStream_t s = (cudaStream_t)stream;
    PVT_CK(cudaMemcpyAsync(orow, dag->orow, (size_t)(dag->n + 1) * sizeof(int64_t), cudaMemcpyDeviceToDevice, s));
    if (dag->m > 0)
        PVT_CK(cudaMemcpyAsync(ocol, dag->ocol, (size_t)dag->m * sizeof(uint32_t), cudaMemcpyDeviceToDevice, s));
    PVT_CK(cudaStreamSynchronize(s));
    return PVT_OK;
}

pvt_status pvt_dag_leaf_depths(pvt_dag *dag, uint64_t *depth, void *stream)
{
    return leaf_depths(dag, depth, (cudaStream_t)stream);
}

pvt_status pvt_count_global(pvt_dag *dag, int32_t kmax, int32_t W, uint64_t *C, void *stream)
{
    const HostRange range("pvt_count_global");
    return count_global(dag, kmax, W, C, (cudaStream_t)stream);
}

pvt_status pvt_count_local_vertex(pvt_dag *dag, int32_t kmax, int32_t W, uint64_t *cv, void *stream)
{
    const HostRange range("pvt_count_local_vertex");
    return count_local(dag, kmax, W, cv, false, (cudaStream_t)stream);
}

pvt_status pvt_count_local_edge(pvt_dag *dag, int32_t kmax, int32_t W, uint64_t *ce, void *stream)
{
    const HostRange range("pvt_count_local_edge");
    return count_local(dag, kmax, W, ce, true, (cudaStream_t)stream);
}

pvt_status pvt_count_hist(pvt_dag *dag, int64_t begin, int64_t end, int32_t kmax, uint64_t *hist, void *stream)
{
    const HostRange range("pvt_count_hist");
    return count_hist(dag, begin, end, kmax, hist, (cudaStream_t)stream);
}

pvt_status pvt_combine_hist(pvt_dag *dag, const uint64_t *hist, int32_t kmax, int32_t W, uint64_t *C,
                            void *stream)
{
    const HostRange range("pvt_combine_hist");
    return combine_hist(dag, hist, kmax, W, C, (cudaStream_t)stream);
}

pvt_status pvt_dag_stats(const pvt_dag *dag, pvt_stats *out)
{
    if (!dag || !out) {
        set_error("pvt_dag_stats: NULL argument");
        return PVT_EINVAL;
    }
    *out = dag->stats;
    for (int i = 0; i < NPHASE; ++i) {
        out->ms[i] = 0.f;
        if (!dag->phase_used[i]) continue;
        float ms = 0.f;
        if (cudaEventSynchronize(dag->ev_t1[i]) == cudaSuccess &&
            cudaEventElapsedTime(&ms, dag->ev_t0[i], dag->ev_t1[i]) == cudaSuccess)
            out->ms[i] = ms;
    }
    return PVT_OK;
}

pvt_status pvt_dag_set_profiling(pvt_dag *dag, int32_t enable)
{
    if (!dag) {
        set_error("pvt_dag_set_profiling: NULL dag");
        return PVT_EINVAL;
    }
    dag->profiling = enable != 0;
    return PVT_OK;
}

pvt_status pvt_dag_set_policy(pvt_dag *dag, const pvt_policy *policy)
{
    bool ok = dag && policy && (policy->persistent == 0 || policy->persistent == 1) && policy->chunk >= 1 &&
              policy->chunk <= 32 && (policy->graph == 0 || policy->graph == 1) &&
              (policy->frames == 0 || policy->frames == 1) && policy->wait_limit_us >= 0 &&
              policy->wait_limit_us <= 1000000000 && (policy->lanes == 0 || policy->lanes == 1);
    for (int c = 0; ok && c < NCLASS; ++c) ok = policy->split[c] == 0 || policy->split[c] == 1;
    for (int c = 0; ok && c < NCLASS; ++c) ok = policy->cta[c] == 0 || (policy->cta[c] == 1 && c >= 4);
    ok = ok && (policy->serial == 0 || policy->serial == 1);
    if (!ok) {
        set_error("pvt_dag_set_policy: invalid argument");
        return PVT_EINVAL;
    }
    dag->policy = *policy;
    drop_graph(dag);
    return PVT_OK;
}

pvt_status pvt_dag_get_policy(const pvt_dag *dag, pvt_policy *out)
{
    if (!dag || !out) {
        set_error("pvt_dag_get_policy: NULL argument");
        return PVT_EINVAL;
    }
    *out = dag->policy;
    return PVT_OK;
}

pvt_status pvt_dag_autotune(pvt_dag *dag, int32_t kmax, int32_t W, uint64_t *C, void *stream,
                            pvt_policy *chosen, float *ms)
{
    const HostRange range("pvt_dag_autotune");
    return autotune(dag, kmax, W, C, (cudaStream_t)stream, chosen, ms);
}

void pvt_dag_free(pvt_dag *dag) { dag_release(dag); }

const char *pvt_last_error(void) { return t_error.c_str(); }

}  // extern "C"
