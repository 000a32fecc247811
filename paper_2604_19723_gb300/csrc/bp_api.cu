// C ABI of libbp (include/bp.h): handle management, validation, launches.
#include <cstdio>
#include <cstring>
#include <cmath>
#include <string>
#include <vector>
#include <algorithm>

#include <nvtx3/nvToolsExt.h>

#include "bp_handle.cuh"

using namespace bp;

static std::string g_init_error;

static bp_status fail(bp_handle* h, bp_status s, const std::string& msg) {
    if (h) h->err = msg; else g_init_error = msg;
    return s;
}

static bp_status cuda_check(bp_handle* h, const char* where) {
    const cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return fail(h, BP_ERR_CUDA, std::string(where) + ": " + cudaGetErrorString(e));
    return BP_OK;
}

template <typename T>
static bool dalloc(bp_handle* h, T** p, size_t count) {
    void* q = nullptr;
    if (cudaMalloc(&q, std::max<size_t>(count, 1) * sizeof(T)) != cudaSuccess) return false;
    h->dev_bytes += std::max<size_t>(count, 1) * sizeof(T);
    cudaMemsetAsync(q, 0, std::max<size_t>(count, 1) * sizeof(T), h->st);
    h->allocs.push_back(q);
    *p = static_cast<T*>(q);
    return true;
}

// stage boundaries: CUDA events when profiling is on, and NVTX ranges (named like the
// profile stages) around the launches of each stage for tools that attach
static const char* const kStageNames[BP_PROF_STAGES] = {"bp.predict", "bp.row_sums", "bp.table", "bp.stage",
                                                        "bp.kappa",   "bp.iota",     "bp.nu",    "bp.normalize",
                                                        "bp.resample"};
static void mark(bp_handle* h, int stage) {
    if (h->prof_on) cudaEventRecord(h->ev[stage], h->st);
    if (h->nvtx_open) nvtxRangePop();
    nvtxRangePushA(kStageNames[stage]);
    h->nvtx_open = true;
}
static void mark_end(bp_handle* h) {
    if (h->nvtx_open) nvtxRangePop();
    h->nvtx_open = false;
}

static int sc_bucket(int S) { return S <= 8 ? 8 : S <= 16 ? 16 : S <= 32 ? 32 : 64; }

bp_status validate_geom(const bp_geometry* g) {
    if (!g || !g->p_pa || !g->R_pa || !g->p_y || !g->p_z) return BP_ERR_INVALID_ARG;
    if (g->J < 1 || g->J > J_MAX || g->Nf < 1 || g->Nf > NF_MAX || g->My < 1 || g->My > MY_MAX || g->Mz < 1 ||
        g->Mz > MZ_MAX || g->Nf * g->My * g->Mz > NZ_MAX)
        return BP_ERR_INVALID_ARG;
    if (!(g->fc > 0) || !(g->c > 0) || !(g->B >= 0)) return BP_ERR_INVALID_ARG;
    return BP_OK;
}

void fill_geom(DevGeom& G, const bp_geometry* g) {
    memset(&G, 0, sizeof(G));
    G.J = g->J; G.Nf = g->Nf; G.My = g->My; G.Mz = g->Mz; G.Nz = g->Nf * g->My * g->Mz;
    G.fc = g->fc; G.c = g->c; G.B = g->B; G.lam = g->c / g->fc;
    for (int j = 0; j < g->J; ++j) {
        for (int k = 0; k < 3; ++k) {
            G.p_pa[j][k] = g->p_pa[3 * j + k];
            G.pa_h[j][k] = (float)G.p_pa[j][k];
            G.pa_l[j][k] = (float)(G.p_pa[j][k] - (double)G.pa_h[j][k]);
        }
        for (int k = 0; k < 9; ++k) {
            G.R[j][k] = g->R_pa[9 * j + k];
            G.R_h[j][k] = (float)G.R[j][k];
            G.R_l[j][k] = (float)(G.R[j][k] - (double)G.R_h[j][k]);
        }
    }
    for (int f = 0; f < g->Nf; ++f) G.f[f] = (g->Nf == 1) ? 0.0 : -0.5 * g->B + f * (g->B / (g->Nf - 1));
    for (int y = 0; y < g->My; ++y) G.py[y] = g->p_y[y];
    for (int m = 0; m < g->Mz; ++m) G.pz[m] = g->p_z[m];
    // float-float constants for the phase reductions (cycles)
    const double il = 1.0 / G.lam;
    G.inv_lam_hi = (float)il;
    G.inv_lam_lo = (float)(il - (double)G.inv_lam_hi);
    for (int f = 0; f < g->Nf; ++f) {
        const double v = G.f[f] / G.c;
        G.fc_hi[f] = (float)v;
        G.fc_lo[f] = (float)(v - (double)G.fc_hi[f]);
    }
    for (int y = 0; y < g->My; ++y) {
        const double v = G.py[y] / G.lam;
        G.py_l[y] = (float)v;
        G.py_lo[y] = (float)(v - (double)G.py_l[y]);
    }
    for (int m = 0; m < g->Mz; ++m) {
        const double v = G.pz[m] / G.lam;
        G.pz_l[m] = (float)v;
        G.pz_lo[m] = (float)(v - (double)G.pz_l[m]);
    }
    G.amp_c = (float)(G.lam / (4.0 * M_PI));
}

extern "C" {

const char* bp_last_error(const bp_handle* h) { return h ? h->err.c_str() : g_init_error.c_str(); }

long long bp_launch_count(const bp_handle* h) { return h ? h->launches : 0; }

bp_status bp_init(const bp_geometry* geom, const bp_params* prm, int P, int S_max, uint64_t seed,
                  void* cuda_stream, bp_handle** out) {
    std::string err;
    const bp_status s = handle_create(geom, prm, P, S_max, 1, seed, static_cast<cudaStream_t>(cuda_stream), true, out, &err);
    if (s != BP_OK) g_init_error = err;
    return s;
}

bp_status bp_free(bp_handle* h) {
    if (!h) return BP_ERR_INVALID_ARG;
    if (h->st) cudaStreamSynchronize(h->st); else cudaDeviceSynchronize();
    if (h->st_side) {
        cudaStreamSynchronize(h->st_side);
        cudaStreamDestroy(h->st_side);
    }
    if (h->ev_fork) cudaEventDestroy(h->ev_fork);
    if (h->ev_join) cudaEventDestroy(h->ev_join);
    if (h->prof_on) for (int i = 0; i <= BP_PROF_STAGES; ++i) cudaEventDestroy(h->ev[i]);
    for (void* p : h->allocs) cudaFree(p);
    if (h->ws_owned && h->ws_base) cudaFree(h->ws_base);
    if (h->h_ctrl) cudaFreeHost(h->h_ctrl);
    if (h->h_est) cudaFreeHost(h->h_est);
    delete h;
    return BP_OK;
}

bp_status bp_predict(bp_handle* h) {
    if (!h) return BP_ERR_INVALID_ARG;
    if (h->phase != 0) return fail(h, BP_ERR_STATE, "bp_predict: the handle already holds a prediction");
    predict_enqueue(h);
    return cuda_check(h, "bp_predict");
}

bp_status bp_update(bp_handle* h, const float* z_dev) {
    if (!h || !z_dev) return BP_ERR_INVALID_ARG;
    if (h->phase != 1) return fail(h, BP_ERR_STATE, "bp_update: call bp_predict (or bp_set_predicted) first");
    if (!h->ws_base) return fail(h, BP_ERR_STATE, "bp_update: no workspace bound");
    update_enqueue(h, z_dev);
    bp_status s = cuda_check(h, "bp_update");
    if (s != BP_OK) return s;
    if (dynamic_pf_count(h)) {
        if (cudaStreamSynchronize(h->st) != cudaSuccess)
            return fail(h, BP_ERR_CUDA, std::string("bp_update: ") + cudaGetErrorString(cudaGetLastError()));
        update_finish(h);
    }
    return BP_OK;
}

bp_status bp_estimate(bp_handle* h, bp_estimate_out* o) {
    if (!h || !o) return BP_ERR_INVALID_ARG;
    const EstLayout E{h->S_max, h->J};
    // h_ctrl has room for S_max more ints; its last slot receives the kernels' timeout flag
    int* kerr_host = h->h_ctrl + 3 + h->S_max;
    if (cudaMemcpyAsync(h->h_est, h->D.est, E.total() * sizeof(double), cudaMemcpyDeviceToHost, h->st) != cudaSuccess ||
        cudaMemcpyAsync(kerr_host, h->D.kerr, sizeof(int), cudaMemcpyDeviceToHost, h->st) != cudaSuccess ||
        cudaStreamSynchronize(h->st) != cudaSuccess)
        return fail(h, BP_ERR_CUDA, std::string("bp_estimate: ") + cudaGetErrorString(cudaGetLastError()));
    if (*kerr_host != 0) {
        const int k = *kerr_host;
        cudaMemsetAsync(h->D.kerr, 0, sizeof(int), h->st);
        if (k & KERR_INDEX)
            return fail(h, BP_ERR_STATE, "bp_estimate: a device index check failed in the last step (checked build)");
        return fail(h, BP_ERR_TIMEOUT, "bp_estimate: a tensor-core wait of the last update gave up (results invalid)");
    }
    const double* e = h->h_est;
    o->n = (int)e[E.n()];
    o->S = (int)e[E.S()];
    o->S_next = (int)e[E.S_next()];
    o->births_skipped = h->births_skipped;
    for (int k = 0; k < 6; ++k) o->x_hat[k] = e[E.x_hat() + k];
    o->ess_x = e[E.ess()];
    o->iota_repaired = (int)e[E.repaired()];
    const int S = o->S;
    if (o->eta_hat) for (int j = 0; j < h->J; ++j) o->eta_hat[j] = e[E.eta_hat() + j];
    if (o->p_s) for (int s = 0; s < S; ++s) o->p_s[s] = e[E.p_s() + s];
    if (o->phi_hat) for (int s = 0; s < 6 * S; ++s) o->phi_hat[s] = e[E.phi_hat() + s];
    if (o->p_pr) for (int s = 0; s < S * h->J; ++s) o->p_pr[s] = e[E.p_pr() + s];
    if (o->declared) for (int s = 0; s < S; ++s) o->declared[s] = e[E.declared() + s] != 0.0;
    if ((int)e[E.status()] == EST_STATUS_BAD_Z)
        return fail(h, BP_ERR_NUMERIC, "the observation of the last update holds NaN or Inf (the state is invalid)");
    if ((int)e[E.status()] == BP_ERR_NUMERIC) return fail(h, BP_ERR_NUMERIC, "all MT weights underflowed");
    return BP_OK;
}

static bp_status copy_state(bp_handle* h, bp_state_view* v, bool to_host, bool predicted) {
    if (!h || !v) return BP_ERR_INVALID_ARG;
    const int P = h->P, J = h->J;
    const cudaMemcpyKind kind = to_host ? cudaMemcpyDeviceToHost : cudaMemcpyHostToDevice;
    int S = to_host ? h->S : v->S;
    if (S < 1 || S > h->S_max) return fail(h, BP_ERR_INVALID_ARG, "S out of range");
    DevState& D = h->D;
    double* wy = predicted ? D.w_alpha : D.w_y;
    double* pr = predicted ? D.zeta : D.p_pr;
    struct Item { void* dev; void* host; size_t bytes; };
    const Item items[] = {
        {D.x[D.cur], v->x, 6 * (size_t)P * sizeof(float)},
        {D.phi[D.cur], v->phi, (size_t)S * 6 * P * sizeof(float)},
        {D.eta[D.cur], v->eta, (size_t)J * P * sizeof(float)},
        {D.w_x, v->w_x, (size_t)P * sizeof(double)},
        {wy, v->w_y, (size_t)S * P * sizeof(double)},
        {D.w_eta, v->w_eta, (size_t)J * P * sizeof(double)},
        {pr, v->p_pr, (size_t)S * J * sizeof(double)},
    };
    for (const Item& it : items) {
        if (!it.host) return fail(h, BP_ERR_INVALID_ARG, "state view has a NULL array");
        cudaError_t e = to_host ? cudaMemcpyAsync(it.host, it.dev, it.bytes, kind, h->st)
                                : cudaMemcpyAsync(it.dev, it.host, it.bytes, kind, h->st);
        if (e != cudaSuccess) return fail(h, BP_ERR_CUDA, cudaGetErrorString(e));
    }
    if (!to_host) {
        // the device step index follows the imported state (pageable copy: staged before return)
        const int nstep = v->n;
        if (cudaMemcpyAsync(D.step, &nstep, sizeof(int), cudaMemcpyHostToDevice, h->st) != cudaSuccess)
            return fail(h, BP_ERR_CUDA, cudaGetErrorString(cudaGetLastError()));
    }
    if (cudaStreamSynchronize(h->st) != cudaSuccess) return fail(h, BP_ERR_CUDA, cudaGetErrorString(cudaGetLastError()));
    if (to_host) { v->S = h->S; v->n = h->n; v->S_legacy = predicted ? h->S_legacy : h->S; }
    else {
        h->S = S;
        // an imported prediction names its new PFs (their birth proposal runs in bp_update)
        h->S_legacy = (predicted && v->S_legacy > 0 && v->S_legacy < S) ? v->S_legacy : S;
        h->n = v->n;
        h->phase = predicted ? 1 : 0;
    }
    return BP_OK;
}

bp_status bp_get_state(bp_handle* h, bp_state_view* out) {
    if (h && h->phase != 0) return fail(h, BP_ERR_STATE, "bp_get_state: the handle holds a prediction");
    return copy_state(h, out, true, false);
}
bp_status bp_set_state(bp_handle* h, const bp_state_view* in) { return copy_state(h, const_cast<bp_state_view*>(in), false, false); }
bp_status bp_get_predicted(bp_handle* h, bp_state_view* out) {
    if (h && h->phase != 1) return fail(h, BP_ERR_STATE, "bp_get_predicted: no prediction held");
    return copy_state(h, out, true, true);
}
bp_status bp_set_predicted(bp_handle* h, const bp_state_view* in) { return copy_state(h, const_cast<bp_state_view*>(in), false, true); }

bp_status bp_get_diag(bp_handle* h, int what, void* host, size_t bytes) {
    if (!h || !host) return BP_ERR_INVALID_ARG;
    if (h->ws_shared) return fail(h, BP_ERR_STATE, "bp_get_diag: the handle's workspace is shared within a batch");
    const int S = h->S_upd, J = h->J, P = h->P, Nz = h->Nz, SM = h->S_max;
    DevState& D = h->D;
    std::vector<std::pair<const void*, size_t>> parts;   // (device ptr, bytes) in order
    if (what == BP_DIAG_TABLE) {
        const size_t plane = (size_t)SM * J * Nz * 2;
        for (int i = 0; i < 4; ++i) parts.push_back({D.tab + i * plane, (size_t)S * J * Nz * 2 * sizeof(double)});
        parts.push_back({D.W, (size_t)S * sizeof(double)});
        parts.push_back({D.eta_bar, (size_t)J * sizeof(double)});
    } else if (what == BP_DIAG_WEIGHTS) {
        parts.push_back({h->wn, (size_t)P * sizeof(double)});
        parts.push_back({h->wn + P, (size_t)S * P * sizeof(double)});
        parts.push_back({h->wn + (size_t)(1 + SM) * P, (size_t)J * P * sizeof(double)});
        parts.push_back({D.p_s, (size_t)S * sizeof(double)});
        parts.push_back({D.bel + BEL_PPR, (size_t)S * J * sizeof(double)});
    } else if (what == BP_DIAG_LOGLIK) {
        parts.push_back({D.lw_x, (size_t)P * sizeof(double)});
        parts.push_back({D.lw_y, (size_t)S * P * sizeof(double)});
        parts.push_back({D.lw_eta, (size_t)J * P * sizeof(double)});
        parts.push_back({D.llr_w, (size_t)S * J * sizeof(double)});
    } else if (what == BP_DIAG_PROPOSAL) {
        const int Qe = S - h->S_legacy;
        if (!D.bprop || Qe < 1) return fail(h, BP_ERR_STATE, "bp_get_diag: no birth proposal in the last update");
        const BpropLayout B = bprop_layout(h->G, h->Pm);
        const size_t Ng = (size_t)h->Pm.N_g;
        parts.push_back({D.bprop + B.stats(0), (size_t)Qe * 32 * sizeof(double)});
        parts.push_back({D.bprop + B.costs(), (size_t)Qe * Ng * sizeof(double)});
        parts.push_back({D.bprop + B.cand(), (size_t)Qe * Ng * 3 * sizeof(double)});
        parts.push_back({D.w_alpha + (size_t)h->S_legacy * P, (size_t)Qe * P * sizeof(double)});
        // the predicted particles stay in the buffer the update resampled from
        const float* pred_phi = D.phi[1 - D.cur];
        for (int s = h->S_legacy; s < S; ++s) parts.push_back({pred_phi + (size_t)s * 6 * P, (size_t)3 * P * sizeof(float)});
    } else if (what == BP_DIAG_LPROP) {
        if (!h->lp_net || !h->lp_buf) return fail(h, BP_ERR_STATE, "bp_get_diag: no proposal network attached");
        parts.push_back({h->lp_buf, (size_t)(6 + 4 * J) * sizeof(double)});
        parts.push_back({h->lp_logr, (size_t)P * sizeof(double)});
        parts.push_back({h->lp_X, (size_t)P * 16 * sizeof(float)});
        parts.push_back({h->lp_Y, (size_t)P * 16 * sizeof(float)});
    } else if (what == BP_DIAG_IOTA) {
        parts.push_back({D.flags, (size_t)(P + 1) * sizeof(int)});
        parts.push_back({D.iota_err, (size_t)P * sizeof(float)});
    } else if (what == BP_DIAG_INDICES) {
        parts.push_back({D.idx, (size_t)P * sizeof(int)});
        parts.push_back({D.idx + P, (size_t)S * P * sizeof(int)});
        parts.push_back({D.idx + (size_t)(1 + SM) * P, (size_t)J * P * sizeof(int)});
    } else {
        return fail(h, BP_ERR_INVALID_ARG, "unknown diagnostic");
    }
    size_t need = 0;
    for (auto& pr : parts) need += pr.second;
    if (bytes < need) return fail(h, BP_ERR_INVALID_ARG, "diagnostic buffer too small");
    char* dst = static_cast<char*>(host);
    for (auto& pr : parts) {
        if (cudaMemcpyAsync(dst, pr.first, pr.second, cudaMemcpyDeviceToHost, h->st) != cudaSuccess)
            return fail(h, BP_ERR_CUDA, cudaGetErrorString(cudaGetLastError()));
        dst += pr.second;
    }
    if (cudaStreamSynchronize(h->st) != cudaSuccess) return fail(h, BP_ERR_CUDA, cudaGetErrorString(cudaGetLastError()));
    return BP_OK;
}

bp_status bp_set_tiles(bp_handle* h, const bp_tiles* t) {
    if (!h || !t) return BP_ERR_INVALID_ARG;
    const int sc = t->kappa_sc;
    const bool ok = (sc == 0 || sc == 8 || sc == 16 || sc == 24 || sc == 32 || sc == 48 || sc == 64) &&
                    (t->kappa_blocks == 0 || t->kappa_blocks == 1 || t->kappa_blocks == 2) && t->kappa_fch >= 0 &&
                    (t->kappa_tc == 0 || t->kappa_tc == 1 || t->kappa_tc == -1) &&
                    (t->table_chunk == 0 || t->table_chunk == 16 || t->table_chunk == 32 || t->table_chunk == 64 ||
                     t->table_chunk == 128) &&
                    t->table_split >= 0;
    if (!ok) return fail(h, BP_ERR_INVALID_ARG, "bp_set_tiles: a field is outside its list of values");
    h->tiles = *t;
    return BP_OK;
}

bp_status bp_get_tiles(const bp_handle* h, bp_tiles* t) {
    if (!h || !t) return BP_ERR_INVALID_ARG;
    *t = h->tiles;
    return BP_OK;
}

bp_status bp_set_profiling(bp_handle* h, int on) {
    if (!h) return BP_ERR_INVALID_ARG;
    if (on && !h->prof_on) {
        for (int i = 0; i <= BP_PROF_STAGES; ++i)
            if (cudaEventCreate(&h->ev[i]) != cudaSuccess) return fail(h, BP_ERR_CUDA, "cudaEventCreate failed");
        for (int i = 0; i < BP_PROF_STAGES; ++i) h->ev_valid[i] = false;
        h->prof_on = 1;
    } else if (!on && h->prof_on) {
        cudaStreamSynchronize(h->st);
        for (int i = 0; i <= BP_PROF_STAGES; ++i) cudaEventDestroy(h->ev[i]);
        h->prof_on = 0;
    }
    return BP_OK;
}

// durations of the last predict (stage 0) and update (stages 1..8); a stage ends
// where the next one starts (the update's last stage ends at the closing event)
bp_status bp_get_profile(bp_handle* h, double* ms, int n) {
    if (!h || !ms || n < BP_PROF_STAGES) return BP_ERR_INVALID_ARG;
    if (!h->prof_on) return fail(h, BP_ERR_STATE, "profiling is off");
    if (cudaStreamSynchronize(h->st) != cudaSuccess) return fail(h, BP_ERR_CUDA, cudaGetErrorString(cudaGetLastError()));
    for (int i = 0; i < BP_PROF_STAGES; ++i) ms[i] = 0.0;
    // the predict's end event is shared with the update's end: only valid if the
    // update has not been recorded after it, so report predict through stage 1's start
    for (int i = 1; i < BP_PROF_STAGES; ++i) {
        if (!h->ev_valid[i]) continue;
        float t = 0.f;
        cudaEvent_t e1 = (i + 1 < BP_PROF_STAGES) ? h->ev[i + 1] : h->ev[BP_PROF_STAGES];
        if (cudaEventElapsedTime(&t, h->ev[i], e1) == cudaSuccess) ms[i] = t;
    }
    if (h->ev_valid[0] && h->ev_valid[1]) {
        float t = 0.f;
        if (cudaEventElapsedTime(&t, h->ev[0], h->ev[1]) == cudaSuccess) ms[0] = t;
    }
    cudaGetLastError();
    return BP_OK;
}

bp_status bp_synthesize(const bp_geometry* geom, int n_steps, int step0, const double* x_pos, int K,
                        const double* sfv, const double* rho, const int* clutter_count, const double* clutter_sfv,
                        const double* clutter_rho, double snr_db, uint64_t seed, float* z_dev, double* eta_out,
                        void* cuda_stream) {
    if (validate_geom(geom) != BP_OK || n_steps < 1 || K < 0 || !x_pos || !rho || !z_dev || !eta_out ||
        (K > 0 && !sfv))
        return fail(nullptr, BP_ERR_INVALID_ARG, "bp_synthesize: invalid arguments");
    DevGeom G;
    fill_geom(G, geom);
    cudaStream_t st = static_cast<cudaStream_t>(cuda_stream);
    const int J = G.J, Nz = G.Nz;
    std::vector<int> off(n_steps + 1, 0);
    for (int t = 0; t < n_steps; ++t) off[t + 1] = off[t] + (clutter_count ? clutter_count[t] : 0);
    const int nc = off[n_steps];
    double *dx = nullptr, *dsfv = nullptr, *drho = nullptr, *dcs = nullptr, *dcr = nullptr, *dz = nullptr, *dpow = nullptr;
    int *doff = nullptr, *dzero = nullptr;
    std::vector<void*> tmp;
    auto alloc = [&](void** p, size_t b) { if (cudaMalloc(p, std::max<size_t>(b, 8)) != cudaSuccess) return false; tmp.push_back(*p); return true; };
    bool ok = alloc((void**)&dx, 3 * sizeof(double) * n_steps) && alloc((void**)&dsfv, 3 * sizeof(double) * std::max(K, 1)) &&
              alloc((void**)&drho, 2 * sizeof(double) * (size_t)n_steps * J * (K + 1)) &&
              alloc((void**)&dcs, 3 * sizeof(double) * std::max(nc, 1)) && alloc((void**)&dcr, 2 * sizeof(double) * std::max(nc, 1) * J) &&
              alloc((void**)&dz, 2 * sizeof(double) * (size_t)n_steps * J * Nz) && alloc((void**)&dpow, sizeof(double)) &&
              alloc((void**)&doff, sizeof(int) * (n_steps + 1)) && alloc((void**)&dzero, sizeof(int) * 2);
    double eta = 0.0;
    if (ok) {
        cudaMemcpyAsync(dx, x_pos, 3 * sizeof(double) * n_steps, cudaMemcpyHostToDevice, st);
        if (K > 0) cudaMemcpyAsync(dsfv, sfv, 3 * sizeof(double) * K, cudaMemcpyHostToDevice, st);
        cudaMemcpyAsync(drho, rho, 2 * sizeof(double) * (size_t)n_steps * J * (K + 1), cudaMemcpyHostToDevice, st);
        if (nc > 0) {
            cudaMemcpyAsync(dcs, clutter_sfv, 3 * sizeof(double) * nc, cudaMemcpyHostToDevice, st);
            cudaMemcpyAsync(dcr, clutter_rho, 2 * sizeof(double) * nc * J, cudaMemcpyHostToDevice, st);
        }
        cudaMemcpyAsync(doff, off.data(), sizeof(int) * (n_steps + 1), cudaMemcpyHostToDevice, st);
        cudaMemsetAsync(dzero, 0, sizeof(int) * 2, st);
        // sum-channel power of the first step from the true components only
        launch_synth(G, 1, step0, dx, K, dsfv, drho, dzero, dcs, dcr, dz, 0, 0, st);
        launch_power(G, dz, dpow, st);
        double pch = 0.0;
        cudaMemcpyAsync(&pch, dpow, sizeof(double), cudaMemcpyDeviceToHost, st);
        cudaStreamSynchronize(st);
        eta = pch / pow(10.0, snr_db / 10.0);
        launch_synth(G, n_steps, step0, dx, K, dsfv, drho, doff, dcs, dcr, dz, 0, 0, st);
        launch_synth_noise(G, n_steps, step0, dz, eta, (uint32_t)(seed & 0xFFFFFFFFu), (uint32_t)(seed >> 32), z_dev, st);
        ok = cudaStreamSynchronize(st) == cudaSuccess && cudaGetLastError() == cudaSuccess;
    }
    for (void* p : tmp) cudaFree(p);
    if (!ok) return fail(nullptr, BP_ERR_CUDA, std::string("bp_synthesize: ") + cudaGetErrorString(cudaGetLastError()));
    *eta_out = eta;
    return BP_OK;
}

}  // extern "C"

// ---------------------------------------------------------------- handle internals

static size_t ws_align(size_t b) { return (std::max<size_t>(b, 8) + 255) & ~(size_t)255; }

WsPlan ws_plan(const DevGeom& G, const DevParams& Pm, int SCA, int nsplit_max) {
    const int P = Pm.P, S_max = Pm.S_max;
    WsPlan w{};
    size_t o = 0;
    auto take = [&](size_t bytes) { const size_t at = o; o += ws_align(bytes); return at; };
    const size_t PP = (size_t)P, J = (size_t)G.J, Nz = (size_t)G.Nz, SM = (size_t)S_max;
    const size_t nbel = (size_t)bel_count(S_max, G.J);
    w.lw_x = take(PP * sizeof(double));
    w.lw_y = take(SM * PP * sizeof(double));
    w.lw_eta = take(J * PP * sizeof(double));
    w.geo = take(SM * J * PP * sizeof(float4));
    w.geo_lo = take(SM * J * PP * sizeof(float2));
    w.flags = take((PP + 1) * sizeof(int));
    w.isel = take(256 + PP * sizeof(float));
    w.tab = take(4 * SM * J * Nz * 2 * sizeof(double));
    w.tab_part = take((size_t)nsplit_max * 3 * SM * J * Nz * 2 * sizeof(double));
    w.kV = take(SM * J * Nz * (size_t)SCA * sizeof(float2));
    w.kr0l = take(SM * J * Nz * sizeof(float2));
    w.kB = kappa_tc_ok(G, SCA) ? take(kappa_btile_floats(G, S_max, SCA) * sizeof(float)) : take(0);
    w.red_part = take(nbel * 64 * RED_W * 2 * sizeof(double));
    w.gram = take(J * SM * SM * 2 * sizeof(double));
    w.V64 = take(SM * J * Nz * (size_t)SCA * 2 * sizeof(double));
    w.cdf = take(nbel * PP * sizeof(double));
    w.wn = take(nbel * PP * sizeof(double));
    w.idx = take(nbel * PP * sizeof(int));
    const bool bprop = Pm.birth_proposal && Pm.Q > 0;
    const BpropLayout B = bprop_layout(G, Pm);
    w.bprop = take(bprop ? B.r_total() * sizeof(double) : 0);
    w.bprop_c = take(bprop ? B.c_total() * sizeof(double2) : 0);
    w.total = o;
    return w;
}

void ws_bind(bp_handle* h, char* base) {
    const WsPlan& w = h->wsp;
    DevState& D = h->D;
    D.lw_x = reinterpret_cast<double*>(base + w.lw_x);
    D.lw_y = reinterpret_cast<double*>(base + w.lw_y);
    D.lw_eta = reinterpret_cast<double*>(base + w.lw_eta);
    D.geo = reinterpret_cast<float4*>(base + w.geo);
    D.geo_lo = reinterpret_cast<float2*>(base + w.geo_lo);
    D.flags = reinterpret_cast<int*>(base + w.flags);
    D.iota_key = reinterpret_cast<unsigned long long*>(base + w.isel);
    D.iota_err = reinterpret_cast<float*>(base + w.isel + 256);
    D.tab = reinterpret_cast<double*>(base + w.tab);
    D.tab_part = reinterpret_cast<double*>(base + w.tab_part);
    D.kV = reinterpret_cast<float2*>(base + w.kV);
    D.kr0l = reinterpret_cast<float2*>(base + w.kr0l);
    D.kB = kappa_tc_ok(h->G, h->SCA) ? reinterpret_cast<float*>(base + w.kB) : nullptr;
    D.red_part = reinterpret_cast<double*>(base + w.red_part);
    h->gram = reinterpret_cast<double*>(base + w.gram);
    h->V64 = reinterpret_cast<double*>(base + w.V64);
    h->cdf = reinterpret_cast<double*>(base + w.cdf);
    h->wn = reinterpret_cast<double*>(base + w.wn);
    D.idx = reinterpret_cast<int*>(base + w.idx);
    const bool bprop = h->Pm.birth_proposal && h->Pm.Q > 0;
    D.bprop = bprop ? reinterpret_cast<double*>(base + w.bprop) : nullptr;
    D.bprop_c = bprop ? reinterpret_cast<double2*>(base + w.bprop_c) : nullptr;
    const size_t PP = (size_t)h->P;
    D.wn_x = h->wn;
    D.wn_y = h->wn + PP;
    D.wn_eta = h->wn + (size_t)(1 + h->S_max) * PP;
    h->ws_base = base;
}

bp_status handle_create(const bp_geometry* geom, const bp_params* prm, int P, int S_max, int S0, uint64_t seed,
                        cudaStream_t st, bool own_ws, bp_handle** out, std::string* err) {
    auto bad = [&](const char* m) { *err = m; return BP_ERR_INVALID_ARG; };
    if (!out) return bad("out is NULL");
    *out = nullptr;
    if (validate_geom(geom) != BP_OK) return bad("invalid geometry");
    if (!prm) return bad("params is NULL");
    if (P < 1 || P > (1 << 28)) return bad("P out of range");
    if (S_max < 1 || S_max > S_CAP_MAX) return bad("S_max must be in [1, 64]");
    if (S0 < 1 || S0 > S_max) return bad("the initial PF count must be in [1, S_max]");
    if (prm->c_eta < 1.0 || prm->c_gamma < 1.0) return bad("Gamma shapes must be >= 1");
    if (prm->motion_dims != 2 && prm->motion_dims != 3) return bad("motion_dims must be 2 or 3");
    if (prm->Q < 0 || !(prm->T > 0)) return bad("invalid Q or T");
    if (prm->birth_proposal && (prm->N_g < 1 || prm->N_g > 65536)) return bad("N_g must be in [1, 65536]");
    bp_handle* h = new bp_handle();
    h->st = st;
    fill_geom(h->G, geom);
    if (iota_blk_smem_bytes(h->G, S_max) > 227 * 1024) {
        delete h;
        *err = "geometry and S_max need more shared memory than the MT likelihood kernel has (227 KB)";
        return BP_ERR_CAPACITY;
    }
    DevParams& Pm = h->Pm;
    memset(&Pm, 0, sizeof(Pm));
    Pm.T = prm->T; Pm.sigma_v = prm->sigma_v; Pm.motion_dims = prm->motion_dims;
    Pm.c_eta = prm->c_eta; Pm.c_gamma = prm->c_gamma; Pm.sigma_mu = prm->sigma_mu; Pm.sigma_sfv = prm->sigma_sfv;
    Pm.pS = prm->pS; Pm.pS_pr = prm->pS_pr; Pm.pR_pr = prm->pR_pr; Pm.pB_pr = prm->pB_pr; Pm.mu_B = prm->mu_B;
    Pm.Q = prm->Q;
    const double mq = prm->mu_B / std::max(prm->Q, 1);
    Pm.pB = mq / (1.0 + mq);
    Pm.T_dec = prm->T_dec; Pm.T_pru = prm->T_pru; Pm.gamma_max = prm->gamma_max; Pm.mu_max = prm->mu_max;
    Pm.eta_min = prm->eta_min; Pm.eta_max = prm->eta_max;
    for (int k = 0; k < 3; ++k) { Pm.p_min[k] = prm->p_min[k]; Pm.p_max[k] = prm->p_max[k]; Pm.v_max[k] = prm->v_max[k]; }
    Pm.zero_mean = prm->zero_mean; Pm.mvec_scaling = prm->mvec_scaling; Pm.regularize = prm->regularize;
    Pm.birth_proposal = prm->birth_proposal ? 1 : 0;
    Pm.N_g = prm->N_g;
    Pm.key0 = (uint32_t)(seed & 0xFFFFFFFFu); Pm.key1 = (uint32_t)(seed >> 32);
    Pm.P = P; Pm.S_max = S_max;
    h->P = P; h->S_max = S_max; h->J = geom->J; h->Nz = h->G.Nz;
    h->SCA = sc_bucket(S_max);
    h->nsplit_max = 32;
    const int J = geom->J, SCA = h->SCA;
    const size_t PP = (size_t)P;
    DevState& D = h->D;
    memset(&D, 0, sizeof(D));
    bool ok = true;
    // persistent state: particles (two buffers), weights, existence, estimates
    for (int b = 0; b < 2; ++b) {
        ok &= dalloc(h, &D.x[b], 6 * PP);
        ok &= dalloc(h, &D.phi[b], (size_t)S_max * 6 * PP);
        ok &= dalloc(h, &D.eta[b], (size_t)J * PP);
    }
    ok &= dalloc(h, &D.w_x, PP);
    ok &= dalloc(h, &D.w_y, (size_t)S_max * PP);
    ok &= dalloc(h, &D.w_alpha, (size_t)S_max * PP);
    ok &= dalloc(h, &D.w_eta, (size_t)J * PP);
    ok &= dalloc(h, &D.p_pr, (size_t)S_max * J);
    ok &= dalloc(h, &D.zeta, (size_t)S_max * J);
    ok &= dalloc(h, &D.p_s, (size_t)S_max);
    ok &= dalloc(h, &D.llr_w, (size_t)S_max * J);
    ok &= dalloc(h, &D.W, (size_t)S_max);
    ok &= dalloc(h, &D.eta_bar, (size_t)J);
    ok &= dalloc(h, &D.kdl, (size_t)S_max * J * SCA);
    ok &= dalloc(h, &D.kerr, 1);
    ok &= dalloc(h, &D.ky0, (size_t)S_max * J * SCA);
    ok &= dalloc(h, &D.kJ0, (size_t)S_max * J);
    ok &= dalloc(h, &D.nu_T, (size_t)J * 4 * S_max);
    ok &= dalloc(h, &D.nu_c, (size_t)J * 2);
    const int nbel = bel_count(S_max, J);
    ok &= dalloc(h, &D.bel, bel_total(S_max, J));
    ok &= dalloc(h, &D.Lchol, (size_t)nbel * 36);
    ok &= dalloc(h, &D.ctrl, (size_t)4 + S_max);
    ok &= dalloc(h, &D.step, 1);
    const EstLayout E{S_max, J};
    ok &= dalloc(h, &D.est, E.total());
    ok &= dalloc(h, &h->nu_b, (size_t)J * (S_max + 1) * 2);
    h->wsp = ws_plan(h->G, h->Pm, SCA, h->nsplit_max);
    if (ok && own_ws) {
        void* q = nullptr;
        ok &= cudaMalloc(&q, h->wsp.total) == cudaSuccess;
        if (ok) {
            cudaMemsetAsync(q, 0, h->wsp.total, h->st);
            h->ws_owned = true;
            ws_bind(h, static_cast<char*>(q));
        }
        // the side stream of the tridiagonalisation; without it everything runs on st
        if (ok) {
            bool side = cudaStreamCreateWithFlags(&h->st_side, cudaStreamNonBlocking) == cudaSuccess;
            side = side && cudaEventCreateWithFlags(&h->ev_fork, cudaEventDisableTiming) == cudaSuccess;
            side = side && cudaEventCreateWithFlags(&h->ev_join, cudaEventDisableTiming) == cudaSuccess;
            if (!side) {
                if (h->st_side) cudaStreamDestroy(h->st_side);
                if (h->ev_fork) cudaEventDestroy(h->ev_fork);
                if (h->ev_join) cudaEventDestroy(h->ev_join);
                h->st_side = nullptr; h->ev_fork = nullptr; h->ev_join = nullptr;
                cudaGetLastError();
            }
        }
    }
    if (ok) {
        ok &= cudaMallocHost(&h->h_ctrl, (4 + S_max) * sizeof(int)) == cudaSuccess;
        ok &= cudaMallocHost(&h->h_est, E.total() * sizeof(double)) == cudaSuccess;
    }
    if (!ok) {
        *err = "device allocation failed";
        bp_free(h);
        return BP_ERR_CUDA;
    }
    D.cur = 0;
    launch_init(h->G, h->Pm, D, S0, h->st);
    h->launches += 1;
    h->S = S0; h->S_upd = S0; h->n = 0; h->phase = 0;
    if (cudaStreamSynchronize(h->st) != cudaSuccess || cudaGetLastError() != cudaSuccess) {
        *err = std::string("bp_init: ") + cudaGetErrorString(cudaGetLastError());
        bp_free(h);
        return BP_ERR_CUDA;
    }
    *out = h;
    return BP_OK;
}

bool dynamic_pf_count(const bp_handle* h) { return h->Pm.Q > 0 || h->Pm.T_pru > 0.0; }

void predict_enqueue(bp_handle* h) {
    const int S_old = h->S;
    int S_new = S_old;
    if (h->Pm.Q > 0) {
        S_new = std::min(S_old + h->Pm.Q, h->S_max);
        h->births_skipped += S_old + h->Pm.Q - S_new;
    }
    mark(h, 0);
    h->launches += launch_predict(h->G, h->Pm, h->D, S_old, S_new, h->st);
    h->S_legacy = S_old;
    if (h->prof_on) { cudaEventRecord(h->ev[BP_PROF_STAGES], h->st); h->ev_valid[0] = true; }
    h->S = S_new;
    h->n += 1;
    h->phase = 1;
    mark_end(h);
}

void update_enqueue(bp_handle* h, const float* z_dev) {
    const int S = h->S, J = h->J, P = h->P;
    DevState& D = h->D;
    mark(h, 1);
    // the learned MT proposal and births drawn from the proposal need this step's observation
    h->launches += launch_learned_proposal(h, z_dev);
    h->launches += launch_birth_proposal(h->G, h->Pm, D, h->S_legacy, S, z_dev, h->st);
    launch_row_sums(h->Pm, D, S, J, h->st);
    mark(h, 2);
    // the built-in split aims at ~4096 table blocks (several waves of short blocks)
    int nsplit = h->tiles.table_split > 0 ? h->tiles.table_split : std::max(1, (4096 + S * J - 1) / (S * J));
    nsplit = std::min(nsplit, std::max(1, P / 256));
    nsplit = std::min(nsplit, h->nsplit_max);
    launch_geom(h->G, h->Pm, D, S, h->st);
    launch_table(h->G, h->Pm, D, S, nsplit, h->tiles.table_chunk, h->st);
    mark(h, 3);
    launch_stage(h->G, h->Pm, D, S, h->SCA, z_dev, h->gram, h->nu_b, h->V64, h->st, h->st_side, h->ev_fork, h->ev_join);
    const KappaPlan kp = plan_kappa(h->G, D, S, h->SCA, h->tiles.kappa_sc, h->tiles.kappa_blocks, h->tiles.kappa_fch,
                                    h->tiles.kappa_tc);
    if (kp.tc) h->launches += launch_kappa_btile(h->G, D, S, h->SCA, h->st);   // B tiles of the tensor-core kernel
    mark(h, 4);
    launch_kappa(h->G, h->Pm, D, S, h->SCA, kp, h->st);
    mark(h, 5);
    const int iota_launches = launch_iota(h->G, h->Pm, D, S, z_dev, h->st) + 1;
    launch_iota_repair(h->G, h->Pm, D, S, z_dev, h->st);
    mark(h, 6);
    if (h->st_side) cudaStreamWaitEvent(h->st, h->ev_join, 0);   // the tridiagonal forms
    launch_nu(h->G, h->Pm, D, S, h->st);
    mark(h, 7);
    launch_normalize(h->G, h->Pm, D, S, h->st);
    mark(h, 8);
    launch_resample(h->G, h->Pm, D, S, h->cdf, h->st);
    if (h->prof_on) {
        cudaEventRecord(h->ev[BP_PROF_STAGES], h->st);
        for (int i = 1; i < BP_PROF_STAGES; ++i) h->ev_valid[i] = true;
    }
    h->launches += 1 + 3 + 3 + 1 + iota_launches + 1 + 5 + 3;
    h->D.cur = 1 - h->D.cur;
    h->S_upd = S;
    h->phase = 0;
    if (dynamic_pf_count(h)) cudaMemcpyAsync(h->h_ctrl, D.ctrl, 4 * sizeof(int), cudaMemcpyDeviceToHost, h->st);
    mark_end(h);
}

void update_finish(bp_handle* h) {
    if (dynamic_pf_count(h)) h->S = h->h_ctrl[1];
}
