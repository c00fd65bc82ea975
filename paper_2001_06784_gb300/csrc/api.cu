// C ABI entry points of libpivoter (declared in include/pivoter.h).
#include <new>
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

static void dag_release(pvt_dag *g)
{
    if (!g) return;
    cudaStreamSynchronize(0);
    drop_graph(g);
    for (int c = 0; c < NCLASS; ++c) {
        if (g->side[c]) { cudaStreamSynchronize(g->side[c]); cudaStreamDestroy(g->side[c]); }
        if (g->ev_join[c]) cudaEventDestroy(g->ev_join[c]);
    }
    if (g->ev_fork) cudaEventDestroy(g->ev_fork);
    for (int i = 0; i < NPHASE; ++i) {
        if (g->ev_t0[i]) cudaEventDestroy(g->ev_t0[i]);
        if (g->ev_t1[i]) cudaEventDestroy(g->ev_t1[i]);
    }
    cudaDeviceSynchronize();
    cudaFree(g->rnd);
    cudaFree(g->core);
    cudaFree(g->orow);
    cudaFree(g->ocol);
    cudaFree(g->oeid);
    cudaFree(g->roots);
    cudaFree(g->d_err);
    cudaFree(g->d_q);
    cudaFree(g->hist.p);
    cudaFree(g->binom.p);
    for (int c = 0; c < NCLASS; ++c) {
        cudaFree(g->rootbuf[c].p);
        cudaFree(g->qframes[c].p);
        cudaFree(g->qready[c].p);
    }
    cudaFree(g->qctl);
    cudaFree(g->cframes.p);
    for (int c = 0; c < NCLASS; ++c) cudaFree(g->gstack[c].p);
    cudaFree(g->d_stats);
    if (g->h_err) cudaFreeHost(g->h_err);
    if (g->h_stats) cudaFreeHost(g->h_stats);
    delete g;
}

}  // namespace pvt

using namespace pvt;

extern "C" {

pvt_status pvt_orient(int64_t n, int64_t nnz, const int64_t *row_ptr, const uint32_t *col,
                      uint32_t flags, void *stream, pvt_dag **dag_out, int32_t *alpha_out)
{
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
    if (e == cudaSuccess) e = cudaMalloc(&g->d_err, sizeof(unsigned));
    if (e == cudaSuccess) e = cudaMalloc(&g->d_q, 16 * sizeof(unsigned));
    if (e == cudaSuccess) e = cudaMalloc(&g->d_stats, 16 * sizeof(unsigned long long));
    if (e == cudaSuccess) e = cudaMalloc(&g->qctl, NCLASS * 128 * sizeof(uint32_t));
    for (int i = 0; i < NPHASE && e == cudaSuccess; ++i) {
        e = cudaEventCreate(&g->ev_t0[i]);
        if (e == cudaSuccess) e = cudaEventCreate(&g->ev_t1[i]);
    }
    if (e == cudaSuccess) e = cudaMallocHost(&g->h_err, sizeof(unsigned));
    if (e == cudaSuccess) e = cudaMallocHost(&g->h_stats, 16 * sizeof(unsigned long long));
    if (e == cudaSuccess) e = cudaEventCreateWithFlags(&g->ev_fork, cudaEventDisableTiming);
    for (int c = 0; c < NCLASS && e == cudaSuccess; ++c) {
        e = cudaStreamCreateWithFlags(&g->side[c], cudaStreamNonBlocking);
        if (e == cudaSuccess) e = cudaEventCreateWithFlags(&g->ev_join[c], cudaEventDisableTiming);
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

pvt_status pvt_count_global(pvt_dag *dag, int32_t kmax, int32_t W, uint64_t *C, void *stream)
{
    return count_global(dag, kmax, W, C, (cudaStream_t)stream);
}

pvt_status pvt_count_local_vertex(pvt_dag *dag, int32_t kmax, int32_t W, uint64_t *cv, void *stream)
{
    return count_local(dag, kmax, W, cv, false, (cudaStream_t)stream);
}

pvt_status pvt_count_local_edge(pvt_dag *dag, int32_t kmax, int32_t W, uint64_t *ce, void *stream)
{
    return count_local(dag, kmax, W, ce, true, (cudaStream_t)stream);
}

pvt_status pvt_count_hist(pvt_dag *dag, int64_t begin, int64_t end, int32_t kmax, uint64_t *hist, void *stream)
{
    return count_hist(dag, begin, end, kmax, hist, (cudaStream_t)stream);
}

pvt_status pvt_combine_hist(pvt_dag *dag, const uint64_t *hist, int32_t kmax, int32_t W, uint64_t *C,
                            void *stream)
{
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
              (policy->frames == 0 || policy->frames == 1);
    for (int c = 0; ok && c < NCLASS; ++c) ok = policy->split[c] == 0 || policy->split[c] == 1;
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
    return autotune(dag, kmax, W, C, (cudaStream_t)stream, chosen, ms);
}

void pvt_dag_free(pvt_dag *dag) { dag_release(dag); }

const char *pvt_last_error(void) { return t_error.c_str(); }

}  // extern "C"
