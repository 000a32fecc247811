// Batches of independent filters (include/bp.h, "batches"): list scheduling of the
// scenarios over concurrent streams, per-stream shared workspaces, and capture of the
// whole batch step into CUDA graphs.
#include <algorithm>
#include <cstring>
#include <numeric>
#include <string>
#include <vector>

#include "bp_handle.cuh"

using namespace bp;

struct bp_batch {
    std::vector<bp_handle*> h;
    std::vector<int> stream_of;            // scenario -> stream
    std::vector<std::vector<int>> queue;   // stream -> scenarios, in launch order
    std::vector<cudaStream_t> streams;
    std::vector<cudaEvent_t> joined;       // per stream: its part of the step is done
    cudaStream_t origin = nullptr;         // fork / join point, and the stream graphs run on
    bool own_origin = false;
    cudaEvent_t forked = nullptr;
    std::vector<char*> ws;                 // workspaces (per stream or per scenario)
    std::vector<size_t> zoff;
    size_t zfloats = 0;
    bool fixed_S = true;                   // no scenario can change its PF count
    bool use_graph = true;
    cudaGraphExec_t exec[2] = {nullptr, nullptr};   // per particle-buffer parity
    const float* exec_z[2] = {nullptr, nullptr};
    std::vector<int> exec_S[2];                     // per scenario: PF count the graph was captured with
    std::vector<long long> graph_launches[2];       // per scenario: kernels in the captured step
    size_t dev_bytes = 0;
    std::string err;
};

namespace {

std::string g_batch_error;   // last bp_batch_init failure

bp_status bfail(bp_batch* b, bp_status s, const std::string& m) {
    b->err = m;
    return s;
}

// relative cost of one step: the PF likelihood (P J S^2 Nz), the message table
// (P J S Nz) and the MT factorisation (P J S^3)
double step_cost(const bp_scenario& sc) {
    const double P = sc.P, J = sc.geom->J, S = sc.S_max;
    const double Nz = (double)sc.geom->Nf * sc.geom->My * sc.geom->Mz;
    return P * J * (Nz * S * (S + 2.0) + 4.0 * S * S * S) + 1e5;
}

// frees everything the batch holds; safe to call again
void release(bp_batch* b) {
    for (int k = 0; k < 2; ++k) {
        if (b->exec[k]) cudaGraphExecDestroy(b->exec[k]);
        b->exec[k] = nullptr;
    }
    for (bp_handle* h : b->h)
        if (h) bp_free(h);
    b->h.clear();
    for (char* w : b->ws)
        if (w) cudaFree(w);
    b->ws.clear();
    for (cudaEvent_t e : b->joined)
        if (e) cudaEventDestroy(e);
    b->joined.clear();
    if (b->forked) cudaEventDestroy(b->forked);
    b->forked = nullptr;
    for (cudaStream_t s : b->streams)
        if (s) cudaStreamDestroy(s);
    b->streams.clear();
    if (b->origin && b->own_origin) cudaStreamDestroy(b->origin);
    b->origin = nullptr;
}

// every stream waits for the origin; afterwards the origin waits for every stream
void fork_streams(bp_batch* b) {
    cudaEventRecord(b->forked, b->origin);
    for (cudaStream_t s : b->streams) cudaStreamWaitEvent(s, b->forked, 0);
}
void join_streams(bp_batch* b) {
    for (size_t k = 0; k < b->streams.size(); ++k) {
        cudaEventRecord(b->joined[k], b->streams[k]);
        cudaStreamWaitEvent(b->origin, b->joined[k], 0);
    }
}

void enqueue_step(bp_batch* b, const float* z_dev) {
    for (const std::vector<int>& q : b->queue)
        for (int i : q) {
            bp_handle* h = b->h[i];
            predict_enqueue(h);
            update_enqueue(h, z_dev + b->zoff[i]);
        }
}

// host-side bookkeeping of one replayed step (what predict_enqueue + update_enqueue do
// besides launching, for a fixed PF count)
void replay_effects(bp_batch* b, int parity) {
    for (size_t i = 0; i < b->h.size(); ++i) {
        bp_handle* h = b->h[i];
        h->n += 1;
        h->launches += b->graph_launches[parity][i];
        h->D.cur = 1 - h->D.cur;
        h->S_upd = h->S;
        h->phase = 0;
    }
}

bp_status capture(bp_batch* b, int parity, const float* z_dev) {
    if (b->exec[parity]) { cudaGraphExecDestroy(b->exec[parity]); b->exec[parity] = nullptr; }
    std::vector<long long> before(b->h.size());
    for (size_t i = 0; i < b->h.size(); ++i) before[i] = b->h[i]->launches;
    if (cudaStreamBeginCapture(b->origin, cudaStreamCaptureModeRelaxed) != cudaSuccess)
        return bfail(b, BP_ERR_CUDA, std::string("capture: ") + cudaGetErrorString(cudaGetLastError()));
    fork_streams(b);
    enqueue_step(b, z_dev);
    join_streams(b);
    cudaGraph_t g = nullptr;
    const cudaError_t e = cudaStreamEndCapture(b->origin, &g);
    // the capture advanced the host bookkeeping by one step that has not run yet: undo it,
    // the replay below applies it again
    b->graph_launches[parity].resize(b->h.size());
    for (size_t i = 0; i < b->h.size(); ++i) {
        bp_handle* h = b->h[i];
        b->graph_launches[parity][i] = h->launches - before[i];
        h->launches = before[i];
        h->n -= 1;
        h->D.cur = 1 - h->D.cur;
    }
    if (e != cudaSuccess || !g) return bfail(b, BP_ERR_CUDA, std::string("capture: ") + cudaGetErrorString(e));
    const cudaError_t ei = cudaGraphInstantiate(&b->exec[parity], g, 0);
    cudaGraphDestroy(g);
    if (ei != cudaSuccess) {
        b->exec[parity] = nullptr;
        return bfail(b, BP_ERR_CUDA, std::string("graph instantiate: ") + cudaGetErrorString(ei));
    }
    b->exec_z[parity] = z_dev;
    b->exec_S[parity].resize(b->h.size());
    for (size_t i = 0; i < b->h.size(); ++i) b->exec_S[parity][i] = b->h[i]->S;
    return BP_OK;
}

}  // namespace

extern "C" {

const char* bp_batch_last_error(const bp_batch* b) { return b ? b->err.c_str() : g_batch_error.c_str(); }

bp_status bp_batch_init(const bp_scenario* sc, int n, const bp_batch_opts* opts, bp_batch** out) {
    if (!out) return BP_ERR_INVALID_ARG;
    *out = nullptr;
    if (!sc || n < 1) return BP_ERR_INVALID_ARG;
    bp_batch_opts o{32, 1, 1, nullptr};
    if (opts) o = *opts;
    if (o.n_streams == 0) o.n_streams = 32;
    if (o.n_streams < 1 || o.n_streams > 128) return BP_ERR_INVALID_ARG;
    for (int i = 0; i < n; ++i)
        if (!sc[i].geom || !sc[i].params) return BP_ERR_INVALID_ARG;
    bp_batch* b = new bp_batch();
    // on any failure: free what was made, report through bp_batch_last_error(NULL)
    auto abort_init = [&](bp_status s, const std::string& m) {
        release(b);
        delete b;
        g_batch_error = m;
        return s;
    };
    b->use_graph = o.use_graph != 0;
    const int K = std::min(o.n_streams, n);
    bool ok = true;
    if (o.cuda_stream) {
        b->origin = static_cast<cudaStream_t>(o.cuda_stream);
    } else {
        // a blocking stream: a step then also follows work on the legacy default stream
        // (e.g. the copy of the observations)
        ok = cudaStreamCreateWithFlags(&b->origin, cudaStreamDefault) == cudaSuccess;
        b->own_origin = ok;
    }
    ok = ok && cudaEventCreateWithFlags(&b->forked, cudaEventDisableTiming) == cudaSuccess;
    b->streams.resize(K, nullptr);
    b->joined.resize(K, nullptr);
    for (int k = 0; ok && k < K; ++k)
        ok = cudaStreamCreateWithFlags(&b->streams[k], cudaStreamNonBlocking) == cudaSuccess &&
             cudaEventCreateWithFlags(&b->joined[k], cudaEventDisableTiming) == cudaSuccess;
    if (!ok) return abort_init(BP_ERR_CUDA, "stream or event creation failed");
    // longest-processing-time list scheduling: costliest scenario first, onto the stream
    // with the least work so far
    std::vector<int> order(n);
    std::iota(order.begin(), order.end(), 0);
    std::vector<double> cost(n);
    for (int i = 0; i < n; ++i) cost[i] = step_cost(sc[i]);
    std::stable_sort(order.begin(), order.end(), [&](int a, int c) { return cost[a] > cost[c]; });
    std::vector<double> load(K, 0.0);
    b->stream_of.assign(n, 0);
    b->queue.assign(K, {});
    for (int i : order) {
        const int k = (int)(std::min_element(load.begin(), load.end()) - load.begin());
        load[k] += cost[i];
        b->stream_of[i] = k;
        b->queue[k].push_back(i);
    }
    // scenarios (persistent state only), observation offsets
    b->h.assign(n, nullptr);
    b->zoff.resize(n);
    for (int i = 0; i < n; ++i) {
        std::string e;
        const bp_status s = handle_create(sc[i].geom, sc[i].params, sc[i].P, sc[i].S_max, sc[i].S0, sc[i].seed,
                                          b->streams[b->stream_of[i]], false, &b->h[i], &e);
        if (s != BP_OK) return abort_init(s, "scenario " + std::to_string(i) + ": " + e);
        b->zoff[i] = b->zfloats;
        b->zfloats += (size_t)2 * sc[i].geom->J * sc[i].geom->Nf * sc[i].geom->My * sc[i].geom->Mz;
        if (dynamic_pf_count(b->h[i])) b->fixed_S = false;
    }
    for (bp_handle* h : b->h) b->dev_bytes += h->dev_bytes;
    smem_optin();   // looked up once, outside any capture
    // workspaces: one per stream, sized for the largest of its scenarios, or one each
    auto alloc_ws = [&](size_t bytes, cudaStream_t st) -> char* {
        void* q = nullptr;
        if (cudaMalloc(&q, bytes) != cudaSuccess) return nullptr;
        cudaMemsetAsync(q, 0, bytes, st);
        b->dev_bytes += bytes;
        return static_cast<char*>(q);
    };
    if (o.shared_workspace) {
        b->ws.assign(K, nullptr);
        for (int k = 0; ok && k < K; ++k) {
            size_t need = 0;
            for (int i : b->queue[k]) need = std::max(need, b->h[i]->wsp.total);
            b->ws[k] = alloc_ws(need, b->streams[k]);
            ok = b->ws[k] != nullptr;
            for (int i : b->queue[k]) {
                ws_bind(b->h[i], b->ws[k]);
                b->h[i]->ws_shared = b->queue[k].size() > 1;
            }
        }
    } else {
        b->ws.assign(n, nullptr);
        for (int i = 0; ok && i < n; ++i) {
            b->ws[i] = alloc_ws(b->h[i]->wsp.total, b->h[i]->st);
            ok = b->ws[i] != nullptr;
            if (ok) ws_bind(b->h[i], b->ws[i]);
        }
    }
    if (!ok) return abort_init(BP_ERR_CUDA, "workspace allocation failed");
    if (cudaDeviceSynchronize() != cudaSuccess)
        return abort_init(BP_ERR_CUDA, std::string("bp_batch_init: ") + cudaGetErrorString(cudaGetLastError()));
    *out = b;
    return BP_OK;
}

bp_status bp_batch_step(bp_batch* b, const float* z_dev) {
    if (!b || !z_dev || b->h.empty()) return BP_ERR_INVALID_ARG;
    for (bp_handle* h : b->h)
        if (h->phase != 0) return bfail(b, BP_ERR_STATE, "bp_batch_step: a scenario holds a prediction");
    if (b->use_graph && b->fixed_S) {
        const int parity = b->h[0]->D.cur;
        for (bp_handle* h : b->h)
            if (h->D.cur != parity) return bfail(b, BP_ERR_STATE, "bp_batch_step: scenarios out of step");
        bool stale = !b->exec[parity] || b->exec_z[parity] != z_dev;
        for (size_t i = 0; !stale && i < b->h.size(); ++i) stale = b->exec_S[parity][i] != b->h[i]->S;
        if (stale) {
            const bp_status s = capture(b, parity, z_dev);
            if (s != BP_OK) return s;
        }
        // the graph runs on the origin stream: it starts after any work issued on the
        // scenarios' own streams, and those streams then wait for it, so that calls on a
        // scenario's handle (bp_estimate, bp_get_state) see the step
        join_streams(b);
        if (cudaGraphLaunch(b->exec[parity], b->origin) != cudaSuccess)
            return bfail(b, BP_ERR_CUDA, std::string("graph launch: ") + cudaGetErrorString(cudaGetLastError()));
        fork_streams(b);
        replay_effects(b, parity);
        return BP_OK;
    }
    fork_streams(b);
    enqueue_step(b, z_dev);
    join_streams(b);
    const cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return bfail(b, BP_ERR_CUDA, std::string("bp_batch_step: ") + cudaGetErrorString(e));
    if (!b->fixed_S) {
        // one synchronisation for the whole batch; then every scenario's new PF count
        if (cudaStreamSynchronize(b->origin) != cudaSuccess)
            return bfail(b, BP_ERR_CUDA, std::string("bp_batch_step: ") + cudaGetErrorString(cudaGetLastError()));
        for (bp_handle* h : b->h) update_finish(h);
    }
    return BP_OK;
}

size_t bp_batch_z_offset(const bp_batch* b, int i) {
    return (b && i >= 0 && i < (int)b->zoff.size()) ? b->zoff[i] : 0;
}
size_t bp_batch_z_floats(const bp_batch* b) { return b ? b->zfloats : 0; }

bp_status bp_batch_sync(bp_batch* b) {
    if (!b) return BP_ERR_INVALID_ARG;
    bool ok = cudaStreamSynchronize(b->origin) == cudaSuccess;
    for (cudaStream_t s : b->streams) ok &= cudaStreamSynchronize(s) == cudaSuccess;
    if (!ok) return bfail(b, BP_ERR_CUDA, std::string("bp_batch_sync: ") + cudaGetErrorString(cudaGetLastError()));
    return BP_OK;
}

bp_status bp_batch_handle(bp_batch* b, int i, bp_handle** h) {
    if (!b || !h || i < 0 || i >= (int)b->h.size()) return BP_ERR_INVALID_ARG;
    *h = b->h[i];
    return BP_OK;
}

bp_status bp_batch_set_tiles(bp_batch* b, int i, const bp_tiles* t) {
    if (!b || !t || i < 0 || i >= (int)b->h.size()) return BP_ERR_INVALID_ARG;
    const bp_status s = bp_set_tiles(b->h[i], t);
    if (s != BP_OK) return bfail(b, s, "bp_batch_set_tiles: a field is outside its list of values");
    // the captured graphs hold the old launch configurations
    for (int k = 0; k < 2; ++k) {
        if (b->exec[k]) cudaGraphExecDestroy(b->exec[k]);
        b->exec[k] = nullptr;
    }
    return BP_OK;
}

int bp_batch_stream_of(const bp_batch* b, int i) {
    return (b && i >= 0 && i < (int)b->stream_of.size()) ? b->stream_of[i] : -1;
}

size_t bp_batch_device_bytes(const bp_batch* b) { return b ? b->dev_bytes : 0; }

bp_status bp_batch_free(bp_batch* b) {
    if (!b) return BP_ERR_INVALID_ARG;
    cudaDeviceSynchronize();
    release(b);
    delete b;
    return BP_OK;
}

}  // extern "C"
