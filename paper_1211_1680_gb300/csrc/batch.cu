// Batches of maps with uneven band-limit and dilation (see s2let_batch_* in
// include/s2let_gpu.h): one plan per (L, B) group, the whole round trip of all
// groups captured once into a CUDA graph (groups on forked streams) and
// replayed with one graph launch.
#include <cuda_runtime.h>

#include <algorithm>
#include <map>
#include <memory>
#include <new>
#include <utility>
#include <vector>

#include "../../include/s2let_gpu.h"

namespace {

struct Group {
    int L, B, n;
    s2let_plan *plan = nullptr;
    int64_t f_off = 0, wav_off = 0, scal_off = 0;
    int64_t f_elems = 0, wav_elems = 0, scal_elems = 0;
    cudaStream_t stream = nullptr;
    cudaEvent_t done = nullptr;
};

struct GraphEntry {
    const void *f;
    void *fw, *fs, *fo;
    cudaStream_t st;
    cudaGraphExec_t exec;
};

int64_t map_elems(int N, bool cplx) { return (int64_t)N * (2 * N - 1) * (cplx ? 2 : 1); }

}  // namespace

struct s2let_batch {
    int n_maps = 0, flags = 0, J0 = 0;
    bool cplx = false;
    std::vector<Group> groups;
    std::vector<int> map_group, map_index;
    int64_t f_elems = 0, wav_elems = 0, scal_elems = 0;
    cudaEvent_t fork = nullptr;
    std::vector<GraphEntry> graphs;
    ~s2let_batch()
    {
        for (auto &g : graphs) cudaGraphExecDestroy(g.exec);
        for (auto &g : groups) {
            if (g.plan) s2let_plan_destroy(g.plan);
            if (g.stream) cudaStreamDestroy(g.stream);
            if (g.done) cudaEventDestroy(g.done);
        }
        if (fork) cudaEventDestroy(fork);
    }
};

extern "C" {

int s2let_batch_create(s2let_batch **out, int n_maps, const int *L, const int *B, int J_min, int flags)
{
    if (!out) return S2LET_ERR_ARG;
    *out = nullptr;
    if (n_maps < 1 || !L || !B) return S2LET_ERR_ARG;
    std::unique_ptr<s2let_batch> b(new (std::nothrow) s2let_batch());
    if (!b) return S2LET_ERR_ALLOC;
    b->n_maps = n_maps;
    b->flags = flags;
    b->J0 = J_min;
    b->cplx = (flags & S2LET_COMPLEX) != 0;
    std::map<std::pair<int, int>, int> index;
    for (int i = 0; i < n_maps; ++i) {
        const auto key = std::make_pair(L[i], B[i]);
        if (!index.count(key)) {
            index[key] = (int)b->groups.size();
            Group g;
            g.L = L[i];
            g.B = B[i];
            g.n = 0;
            b->groups.push_back(g);
        }
    }
    b->map_group.resize(n_maps);
    b->map_index.resize(n_maps);
    for (int i = 0; i < n_maps; ++i) {
        const int g = index[std::make_pair(L[i], B[i])];
        b->map_group[i] = g;
        b->map_index[i] = b->groups[g].n++;
    }
    for (auto &g : b->groups) {
        int e = s2let_plan_create(&g.plan, g.L, g.B, J_min, flags, g.n);
        if (e) return e;
        int64_t we = 0, se = 0;
        if ((e = s2let_plan_info(g.plan, nullptr, nullptr, &we, &se, nullptr))) return e;
        g.f_elems = map_elems(g.L, b->cplx) * g.n;
        g.wav_elems = we;
        g.scal_elems = se;
        g.f_off = b->f_elems;
        g.wav_off = b->wav_elems;
        g.scal_off = b->scal_elems;
        b->f_elems += g.f_elems;
        b->wav_elems += we;
        b->scal_elems += se;
        if (cudaStreamCreateWithFlags(&g.stream, cudaStreamNonBlocking) != cudaSuccess) return S2LET_ERR_CUDA;
        if (cudaEventCreateWithFlags(&g.done, cudaEventDisableTiming) != cudaSuccess) return S2LET_ERR_CUDA;
    }
    if (cudaEventCreateWithFlags(&b->fork, cudaEventDisableTiming) != cudaSuccess) return S2LET_ERR_CUDA;
    *out = b.release();
    return S2LET_OK;
}

int s2let_batch_destroy(s2let_batch *b)
{
    delete b;
    return S2LET_OK;
}

int s2let_batch_sizes(const s2let_batch *b, int64_t *f_elems, int64_t *wav_elems, int64_t *scal_elems, int *n_groups)
{
    if (!b) return S2LET_ERR_ARG;
    if (f_elems) *f_elems = b->f_elems;
    if (wav_elems) *wav_elems = b->wav_elems;
    if (scal_elems) *scal_elems = b->scal_elems;
    if (n_groups) *n_groups = (int)b->groups.size();
    return S2LET_OK;
}

int s2let_batch_map_layout(const s2let_batch *b, int i, int64_t *f_off, int64_t *scal_off, int *group,
                           int *index_in_group)
{
    if (!b || i < 0 || i >= b->n_maps) return S2LET_ERR_ARG;
    const int g = b->map_group[i], k = b->map_index[i];
    const Group &G = b->groups[g];
    int Ns = 0;
    s2let_plan_info(G.plan, nullptr, nullptr, nullptr, nullptr, &Ns);
    if (f_off) *f_off = G.f_off + map_elems(G.L, b->cplx) * k;
    if (scal_off) *scal_off = G.scal_off + map_elems(Ns, b->cplx) * k;
    if (group) *group = g;
    if (index_in_group) *index_in_group = k;
    return S2LET_OK;
}

int s2let_batch_group_plan(const s2let_batch *b, int g, s2let_plan **plan, int64_t *f_off, int64_t *wav_off,
                           int64_t *scal_off)
{
    if (!b || g < 0 || g >= (int)b->groups.size()) return S2LET_ERR_ARG;
    const Group &G = b->groups[g];
    if (plan) *plan = G.plan;
    if (f_off) *f_off = G.f_off;
    if (wav_off) *wav_off = G.wav_off;
    if (scal_off) *scal_off = G.scal_off;
    return S2LET_OK;
}

int s2let_batch_autotune(s2let_batch *b, void *stream)
{
    if (!b) return S2LET_ERR_ARG;
    for (auto &g : b->groups) {
        const int e = s2let_plan_autotune(g.plan, stream);
        if (e) return e;
    }
    // graphs captured before hold the earlier kernel choices
    for (auto &g : b->graphs) cudaGraphExecDestroy(g.exec);
    b->graphs.clear();
    return S2LET_OK;
}

int s2let_batch_round_trip(s2let_batch *b, const void *f, void *fw, void *fs, void *fo, void *stream)
{
    if (!b || !f || !fw || !fs || !fo) return S2LET_ERR_ARG;
    cudaStream_t st = (cudaStream_t)stream;
    for (auto &e : b->graphs)
        if (e.f == f && e.fw == fw && e.fs == fs && e.fo == fo && e.st == st)
            return cudaGraphLaunch(e.exec, st) == cudaSuccess ? S2LET_OK : S2LET_ERR_CUDA;
    if (!st) return S2LET_ERR_ARG;   // capture needs a non-default stream
    const size_t es = (b->flags & S2LET_PREC_MASK) == S2LET_PREC_FP64 ? 8 : 4;
    // capture: fork every group onto its own stream, join back on `st`
    if (cudaStreamBeginCapture(st, cudaStreamCaptureModeThreadLocal) != cudaSuccess) return S2LET_ERR_CUDA;
    int err = S2LET_OK;
    if (cudaEventRecord(b->fork, st) != cudaSuccess) err = S2LET_ERR_CUDA;
    for (auto &g : b->groups) {
        if (err) break;
        if (cudaStreamWaitEvent(g.stream, b->fork, 0) != cudaSuccess) {
            err = S2LET_ERR_CUDA;
            break;
        }
        const char *fi = (const char *)f + g.f_off * es;
        char *wo = (char *)fw + g.wav_off * es;
        char *so = (char *)fs + g.scal_off * es;
        char *oo = (char *)fo + g.f_off * es;
        if ((err = s2let_analysis(g.plan, fi, wo, so, g.stream))) break;
        if ((err = s2let_synthesis(g.plan, wo, so, oo, g.stream))) break;
        if (cudaEventRecord(g.done, g.stream) != cudaSuccess || cudaStreamWaitEvent(st, g.done, 0) != cudaSuccess)
            err = S2LET_ERR_CUDA;
    }
    cudaGraph_t graph = nullptr;
    const cudaError_t ce = cudaStreamEndCapture(st, &graph);
    if (!err && ce != cudaSuccess) err = S2LET_ERR_CUDA;
    if (err) {
        if (graph) cudaGraphDestroy(graph);
        return err;
    }
    cudaGraphExec_t exec = nullptr;
    const cudaError_t ie = cudaGraphInstantiate(&exec, graph, 0);
    cudaGraphDestroy(graph);
    if (ie != cudaSuccess) return S2LET_ERR_CUDA;
    if (b->graphs.size() >= 8) {
        cudaGraphExecDestroy(b->graphs.front().exec);
        b->graphs.erase(b->graphs.begin());
    }
    b->graphs.push_back({f, fw, fs, fo, st, exec});
    return cudaGraphLaunch(exec, st) == cudaSuccess ? S2LET_OK : S2LET_ERR_CUDA;
}

}  // extern "C"
