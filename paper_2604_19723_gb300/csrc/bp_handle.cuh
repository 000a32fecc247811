// Private definition of the filter handle shared by the single-filter entry points
// (bp_api.cu) and the batch executor (bp_batch.cu).
#pragma once
#include <string>
#include <vector>

#include "../../include/bp.h"
#include "bp_internal.cuh"
#include "bp_kernels.cuh"

// Byte offsets of the per-step workspace of one filter: the buffers whose contents
// live only from the start of a bp_update to the end of the diagnostics read after
// it (geometry records, bases, likelihoods, normalised weights, CDFs, indices).  A
// filter on its own owns one; filters of a batch that run one after another on the
// same stream share one, sized for the largest of them.
struct WsPlan {
    size_t lw_x, lw_y, lw_eta, geo, geo_lo, flags, isel, tab, tab_part, kV, kr0l, kB, red_part, gram, V64, cdf, wn, idx;
    size_t bprop, bprop_c;   // birth proposal scratch (empty unless enabled)
    size_t total;
};

struct bp_handle {
    bp::DevGeom G;
    bp::DevParams Pm;
    bp::DevState D;
    cudaStream_t st;
    // single filters: a side stream for the noise-likelihood tridiagonalisation, which
    // runs beside the PF basis stage (fork after the Gram, join before its consumer)
    cudaStream_t st_side;
    cudaEvent_t ev_fork, ev_join;
    int P, S_max, J, Nz;
    int SCA;            // column stride of the per-(s,j) basis buffers
    int S;              // current number of PFs (host copy)
    int S_legacy;       // PFs before the births of the current prediction
    int S_upd;          // S of the last bp_update
    int n;              // last completed step (state) or current step (predicted); the device holds it too
    int phase;          // 0: belief state, 1: predicted
    int births_skipped;
    int nsplit_max;
    bp_tiles tiles;     // kernel tile requests (bp_set_tiles; zero = built-in)
    long long launches;
    size_t dev_bytes;   // device memory of the handle's own allocations (workspace excluded)
    // per-handle scratch
    double* gram;
    double* nu_b;
    double* V64;
    double* cdf;
    double* wn;         // normalised weights before resampling: w_x (P) | w_y (S_max P) | w_eta (J P)
    int* h_ctrl;        // pinned
    double* h_est;      // pinned
    // per-step workspace (owned, or bound by a batch)
    WsPlan wsp;
    char* ws_base;
    bool ws_owned;
    bool ws_shared;     // bound to a workspace that other filters overwrite: no diagnostics
    // learned MT proposal (attached network, not owned; its buffers are)
    bp_mlp* lp_net;
    float* lp_X;        // P x 16 network inputs
    float* lp_Y;        // P x 16 network outputs
    double* lp_logr;    // P log importance ratios of the last update
    double* lp_buf;     // predicted mean (6), per-PA correlations (4 J)
    int prof_on;
    bool nvtx_open;     // an NVTX stage range is open on this thread
    cudaEvent_t ev[BP_PROF_STAGES + 1];
    bool ev_valid[BP_PROF_STAGES];
    std::vector<void*> allocs;
    std::string err;
};

// creates a handle with its persistent state and S0 PFs at time 0 (the LoS and S0 - 1
// drawn from the birth density); with own_ws it also allocates and binds its
// workspace, otherwise the caller binds one with ws_bind before the first update
bp_status handle_create(const bp_geometry* geom, const bp_params* prm, int P, int S_max, int S0, uint64_t seed,
                        cudaStream_t st, bool own_ws, bp_handle** out, std::string* err);
WsPlan ws_plan(const bp::DevGeom& G, const bp::DevParams& Pm, int SCA, int nsplit_max);
void ws_bind(bp_handle* h, char* base);
// launches of one prediction / one update on the handle's stream (no synchronisation);
// update_enqueue also copies the control words to pinned memory when the PF count can
// change, update_finish (after the stream is synchronised) takes the new count
void predict_enqueue(bp_handle* h);
void update_enqueue(bp_handle* h, const float* z_dev);
void update_finish(bp_handle* h);
bool dynamic_pf_count(const bp_handle* h);
// geometry checks and the device copy of its constants (shared with the PCRLB entry points)
bp_status validate_geom(const bp_geometry* g);
void fill_geom(bp::DevGeom& G, const bp_geometry* g);

// proposal network forward pass on a stream (k_mlp.cu), and the learned MT proposal of
// an update (k_lproposal.cu; returns its launch count, 0 without a network)
void mlp_forward_async(const bp_mlp* net, const float* X, int B, float* Y, cudaStream_t st);
int launch_learned_proposal(const bp_handle* h, const float* z_dev);

