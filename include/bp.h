/*
 * bp.h -- C ABI of the GB300 particle-based BP update for direct multipath SLAM
 * ("Soft-Coherent Direct Multipath SLAM", arXiv 2604.19723).
 *
 * One handle holds one filter: P particles per belief for the mobile terminal
 * (MT) state x_n = [p; v] in R^6, for each potential feature (PF)
 * phi_s = [p_sfv (3), gamma, mu (complex)] and for each physical anchor's (PA)
 * noise variance eta^(j), plus the PR existence probabilities p(r_s^(j) = 1).
 * All device memory is allocated by bp_init and released by bp_free.  Every
 * call is asynchronous on the handle's CUDA stream unless stated otherwise.
 *
 * Conventions
 *   - Complex arrays are interleaved (re, im).  Observations z^(j) are
 *     complex FP32, layout [J][Nf][My][Mz] with flat element index
 *     k = f*(My*Mz) + y*Mz + m (the Kronecker order of Sec. II-B,
 *     eq. unit-modulus-array-response).
 *   - Particles are FP32 structure-of-arrays, weights FP64.
 *   - PF slot 0 is the line-of-sight (LoS) component; its p_sfv is unused.
 *   - Host pointers are read (or written) only during the call.
 *   - No C++ exception crosses this ABI.  Every entry returns a bp_status;
 *     bp_last_error() returns the text of the last failure on a handle.
 *
 * Error behaviour: invalid sizes/pointers -> BP_ERR_INVALID_ARG (nothing
 * launched); CUDA runtime failure -> BP_ERR_CUDA; PF capacity exhausted by
 * births -> the birth is skipped and counted (bp_estimate reports it);
 * all particle weights underflow -> BP_ERR_NUMERIC reported by the next
 * synchronising call (bp_estimate / bp_get_state).
 */
#ifndef BP_H
#define BP_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct bp_handle bp_handle;

typedef enum {
    BP_OK = 0,
    BP_ERR_INVALID_ARG = 1,
    BP_ERR_CUDA = 2,
    BP_ERR_CAPACITY = 3,
    BP_ERR_NUMERIC = 4,
    BP_ERR_TIMEOUT = 5,
    BP_ERR_STATE = 6
} bp_status;

/* Array and signal constants (Sec. II-B).  f_k = -B/2 + k B/(Nf-1).
 * R_pa: J rotation matrices, row-major 3x3, columns = local PA axes in
 * global coordinates (local vector r' = R^T r, eq. rangep).  p_y, p_z:
 * template URA element positions, symmetric about 0.
 * Limits: 1 <= J <= 16, Nf <= 128, My <= 16, Mz <= 16, Nz <= 2048. */
typedef struct {
    int J, Nf, My, Mz;
    double fc, c, B;
    const double* p_pa;   /* J x 3 */
    const double* R_pa;   /* J x 3 x 3 */
    const double* p_y;    /* My */
    const double* p_z;    /* Mz */
} bp_geometry;

/* Filter parameters (Sec. III-B, Sec. V).  motion_dims = 3 (3-D NCV) or 2
 * (planar: z and v_z held).  Q births per step (0 = no birth), T_pru = 0
 * disables pruning.  zero_mean = 1 selects the ZM variant (mu == 0).
 * mvec_scaling = 0 uses the m-vectors exactly as printed in Supplementary
 * Sec. S-V; 1 takes the square root of the existence factors.  regularize
 * = 1 applies the Gaussian-kernel jitter after resampling.
 * birth_proposal = 1 draws the positions of new PFs from the Gaussian proposal
 * of Sec. IV-D ("An Efficient Birth Proposal PDF": residual of the observation
 * after projecting out the LoS and legacy PFs, coherent Bartlett spectrum at
 * N_g candidates uniform in the PF's partition, mode-matched mean and
 * moment-matched covariance, weights 1_P / proposal density); 0 draws them
 * from the birth density f_B.  The proposal needs the observation, so bp_update
 * (not bp_predict) draws those particles.  1 <= N_g <= 65536. */
typedef struct {
    double T, sigma_v;
    int motion_dims;
    double c_eta, c_gamma, sigma_mu, sigma_sfv;
    double pS, pS_pr, pR_pr, pB_pr, mu_B;
    int Q;
    double T_dec, T_pru, gamma_max, mu_max, eta_min, eta_max;
    double p_min[3], p_max[3], v_max[3];
    int zero_mean, mvec_scaling, regularize;
    int birth_proposal, N_g;
} bp_params;

/* Host view of a filter state (bp_get_state / bp_set_state) or of the
 * prediction messages (bp_get_predicted / bp_set_predicted).  Sizes use the
 * handle's P, S_max, J; only the first S PF slots are read or written.
 *   x     6 x P          float   MT particles [px py pz vx vy vz]
 *   phi   S x 6 x P      float   PF particles [px py pz gamma mu_re mu_im]
 *   eta   J x P          float   noise-variance particles
 *   w_x   P              double  belief weights w_x     (predicted: w_beta)
 *   w_y   S x P          double  PF weights, sum = p_s  (predicted: w_alpha)
 *   w_eta J x P          double  eta weights            (predicted: w_xi)
 *   p_pr  S x J          double  p(r_s^(j) = 1)         (predicted: zeta_s^(j)(1)) */
typedef struct {
    int n;      /* index of the last completed step (predicted: current step) */
    int S;      /* number of PFs including the LoS */
    int S_legacy; /* predictions: PFs that existed before this step's births (slots
                     S_legacy .. S-1 are new; 0 or S = none new); states: ignored,
                     written as S */
    float* x;
    float* phi;
    float* eta;
    double* w_x;
    double* w_y;
    double* w_eta;
    double* p_pr;
} bp_state_view;

/* MMSE estimates and declarations (Sec. II-C, eq. stateHat, etanHat,
 * PFphiHat).  Arrays are caller-owned: eta_hat[J], p_s[S_max],
 * phi_hat[S_max*6], p_pr[S_max*J], declared[S_max]. */
typedef struct {
    int n;               /* step the estimate belongs to */
    int S;               /* PFs before pruning (valid entries in the arrays) */
    int S_next;          /* PFs kept for the next step */
    int births_skipped;  /* births dropped because S_max was reached (cumulative) */
    double x_hat[6];
    double ess_x;        /* 1 / sum w_x^2 */
    double* eta_hat;
    double* p_s;
    double* phi_hat;
    double* p_pr;
    int* declared;
    int iota_repaired;   /* particles whose MT likelihood was recomputed in FP64 (ill-conditioned) */
} bp_estimate_out;

/* Creates a filter: validates, copies the geometry and parameters, allocates
 * the device state for P particles per belief and up to S_max PFs
 * (S_max <= 64), and draws the time-0 beliefs of Sec. V-A (MT from the
 * uniform box, eta from U(eta_min, eta_max), the LoS like a new PF).
 * cuda_stream: a cudaStream_t (NULL = legacy default stream).
 * seed selects the Philox4x32-10 key.  Synchronous. */
bp_status bp_init(const bp_geometry* geom, const bp_params* params, int P, int S_max,
                  uint64_t seed, void* cuda_stream, bp_handle** out);

/* Phase (i) of the message schedule (Sec. IV): prediction messages beta, xi,
 * alpha, zeta of every belief (Sec. IV-D, eq. PR-prediction-PDF, eq. zeta)
 * plus Q birth PFs drawn from f_B (Sec. III-B2, IV-D). */
bp_status bp_predict(bp_handle* h);

/* Phases (ii)-(iii) and the belief update (Sec. IV-C/D, Supplementary S-III
 * to S-VI): message table, per-(s,j) existence tests, per-particle
 * likelihoods, FP64 normalisation, estimates, pruning, systematic
 * resampling and regularisation.  z_dev: device pointer to the J x Nz
 * complex FP32 observations of this step, borrowed for the call's
 * duration on the handle's stream. */
bp_status bp_update(bp_handle* h, const float* z_dev);

/* Copies the estimates of the last bp_update to the host.  Synchronous.  Returns
 * BP_ERR_NUMERIC when every MT weight underflowed, or when the observation of the last
 * update held NaN or Inf (bp_last_error says which; the state is then invalid and a
 * checkpoint should be restored), BP_ERR_TIMEOUT when a bounded tensor-core wait of the
 * update gave up. */
bp_status bp_estimate(bp_handle* h, bp_estimate_out* out);

/* Releases every device buffer of the handle.  Synchronous. */
bp_status bp_free(bp_handle* h);

/* Text of the last error on h (or of the last bp_init failure if h is NULL). */
const char* bp_last_error(const bp_handle* h);

/* State export / import (checkpoint and resume, parity tests).  Synchronous. */
bp_status bp_get_state(bp_handle* h, bp_state_view* out);
bp_status bp_set_state(bp_handle* h, const bp_state_view* in);

/* Prediction-message export / import: bp_set_predicted puts the handle in
 * the state reached after bp_predict, so that bp_update runs from the given
 * particles and weights.  Synchronous. */
bp_status bp_get_predicted(bp_handle* h, bp_state_view* out);
bp_status bp_set_predicted(bp_handle* h, const bp_state_view* in);

/* Diagnostics of the last bp_update, copied to host memory (synchronous).
 * what = BP_DIAG_TABLE: S x J x Nz complex double for each of
 *        m, m^w, mu3, mu4 (in that order), then W_s (S), eta_bar (J);
 *        bytes = (4*S*J*Nz*2 + S + J) * 8.
 * what = BP_DIAG_WEIGHTS: normalised weights before resampling:
 *        w_x (P), w_y (S x P), w_eta (J x P), p_s (S), p_pr (S x J), all double.
 * what = BP_DIAG_LOGLIK: particle log-likelihood sums: log iota (P) summed over
 *        j, Delta_kappa (S x P) summed over j (log kappa~(phi,1) - log kappa~(.,0)),
 *        log nu (J x P), log omega~(1)-log omega~(0) (S x J); double.
 * what = BP_DIAG_INDICES: resampling indices, int32: MT (P), PF (S x P), eta (J x P).
 * what = BP_DIAG_PROPOSAL (birth_proposal = 1, new PFs in the last update; Qe =
 *        their number, Ng = N_g): per new PF the statistics [32] doubles (valid,
 *        i*, sum of costs, mu [3], C [3x3], L [3x3], 0-padded), the Bartlett costs
 *        [Qe][Ng] and candidates [Qe][Ng][3] (double), the prediction weights
 *        w_alpha [Qe][P] (double), then the new PFs' particle positions [Qe][3][P]
 *        (float).  BP_ERR_STATE without a proposal in the last update.
 * what = BP_DIAG_LPROP (a proposal network attached): the predicted mean xbar (6) and
 *        the per-PA correlations (Re, Im of psi_j(xbar)^H z_j, |z_j|^2, |psi_j|^2) for
 *        J PAs (double), the log importance ratios (P, double), the network inputs and
 *        outputs (P x 16 each, float).  BP_ERR_STATE without a network.
 * what = BP_DIAG_IOTA (S >= 24 in the last update): the particles evaluated in
 *        float-float, int32 [1 + P] (count, then their indices), and the error bound
 *        (nats) of every particle's FP32 log iota sum, float [P].  The log iota of a
 *        particle not in the list is its FP32 value (BP_DIAG_LOGLIK). */
enum { BP_DIAG_TABLE = 1, BP_DIAG_WEIGHTS = 2, BP_DIAG_LOGLIK = 3, BP_DIAG_INDICES = 4, BP_DIAG_PROPOSAL = 5,
       BP_DIAG_LPROP = 6, BP_DIAG_IOTA = 7 };
bp_status bp_get_diag(bp_handle* h, int what, void* host, size_t bytes);

/* Synthetic observations from the generative model (eq. observation-generative),
 * for tests and benchmarks.  For each of n_steps steps t: MT position
 * x_pos[t*3..], K surfaces with SFVs sfv[K*3] and complex amplitudes
 * rho[((t*J + j)*(K+1) + k)*2] (k = 0 the LoS, 0 for an invisible path),
 * plus clutter_count[t] spurious paths with SFVs clutter_sfv and amplitudes
 * clutter_rho[(c*J + j)*2] (concatenated over t).  The noise variance is
 * eta = P^ch / 10^(snr_db/10) with P^ch the sum-channel power of the first
 * step (Sec. V-A); it is returned in *eta_out.  Noise uses Philox draws of
 * step index step0 + t.  z_dev: device, n_steps x J x Nz complex FP32.
 * Synchronous. */
bp_status bp_synthesize(const bp_geometry* geom, int n_steps, int step0, const double* x_pos,
                        int K, const double* sfv, const double* rho,
                        const int* clutter_count, const double* clutter_sfv, const double* clutter_rho,
                        double snr_db, uint64_t seed, float* z_dev, double* eta_out, void* cuda_stream);

/* Number of kernels launched by this handle since bp_init (instrumentation). */
long long bp_launch_count(const bp_handle* h);

/* Self-test of the bounded device waits that the tensor-core kernels use: one thread
 * waits, at most `limit` polls (1 .. 2^20), on an mbarrier phase that nothing completes.
 * Returns BP_ERR_TIMEOUT (the expected outcome: the wait gave up and the kernel ended
 * normally, the context stays usable), BP_OK if the phase completed, BP_ERR_CUDA on a
 * launch failure.  Synchronous. */
bp_status bp_selftest_wait(int limit, void* cuda_stream);

/* Per-stage timing with CUDA events recorded on the handle's stream
 * (instrumentation, off by default).  bp_get_profile waits for the last
 * bp_predict / bp_update and writes the duration in milliseconds of each
 * stage of those calls into ms[0 .. BP_PROF_STAGES-1]:
 * predict, row sums, message table, table stage (Gram, kappa/omega, nu),
 * kappa likelihood, iota likelihood, nu likelihood, normalisation, resampling. */
enum { BP_PROF_STAGES = 9 };
bp_status bp_set_profiling(bp_handle* h, int on);
bp_status bp_get_profile(bp_handle* h, double* ms, int n);

/* Kernel tile configuration of a filter: the knobs of the measured autotuner
 * (paper_2604_19723_gb300/autotune.py).  The paper has no counterpart; results
 * depend on them only through FP32 rounding.  0 in a field = the built-in
 * choice.
 *   kappa_sc      column bucket S~ of the CUDA-core PF likelihood (S~ - 1 basis
 *                 columns held per particle): 8, 16, 24, 32, 48 or 64.  Used
 *                 when S <= kappa_sc <= the filter's basis stride (32 for
 *                 S_max <= 32, else 64), otherwise the smallest bucket >= S.
 *   kappa_blocks  CUDA-core PF-likelihood blocks of 256 particles per SM: 1 or 2
 *                 (2 caps registers at 128 per thread and shrinks the staged
 *                 frequency chunk; buckets <= 32 only, else 1 is used).
 *   kappa_fch     frequencies of V staged in shared memory per chunk (the Nz
 *                 tile), clamped to what fits.
 *   kappa_tc      1: the tensor-core PF likelihood wherever the shape allows it,
 *                 at the bucket equal to the basis stride (Mz even, and either
 *                 64 basis columns with 2 My Mz in {8, 16, 32}, or 32 or 64
 *                 columns with My Mz a multiple of 16, at least 32; shared
 *                 memory within 227 KB); built-in (0): the same where the
 *                 bucket is the stride; -1: never.
 *   table_chunk   particles per shared-memory chunk of the message table: 16,
 *                 32, 64 or 128 (clamped to what fits; built-in 64).
 *   table_split   particle splits of the message-table grid (>= 1; clamped to
 *                 P / 256 and the workspace's partial-sum capacity; built-in
 *                 about 4096 blocks over the S x J problems).
 * bp_set_tiles validates and stores the fields (BP_ERR_INVALID_ARG for a value
 * outside the lists above; nothing is changed then); they apply from the next
 * bp_update.  bp_get_tiles returns the stored fields.  Host-only calls. */
typedef struct {
    int kappa_sc, kappa_blocks, kappa_fch, kappa_tc, table_chunk, table_split;
} bp_tiles;
bp_status bp_set_tiles(bp_handle* h, const bp_tiles* t);
bp_status bp_get_tiles(const bp_handle* h, bp_tiles* t);

/* Systematic resampling of one belief that allocates no device memory.
 * The paper has no counterpart: this entry point exists for callers that
 * cannot call cudaMalloc (code under CUDA graph capture, real-time loops that
 * forbid allocator calls, hosts whose device memory belongs to another
 * allocator).  It runs the resampler bp_update applies to every belief, with
 * its FP64 cumulative-weight scratch in a static device array of
 * BP_NOALLOC_MAX_P doubles (8 MiB) that every GPU loading the library holds
 * until the process exits.
 *   w_dev   device, P non-negative weights (need not be normalised), read only
 *   P       1 .. BP_NOALLOC_MAX_P; larger P returns BP_ERR_CAPACITY, nothing launched
 *   seed, n, kind, index   select the uniform U exactly as bp_update does for
 *           the belief (kind 0 = MT, 1 = PF slot index, 2 = eta of PA index)
 *           at step n; particle i takes the first k with CDF_k >= (U + i)/P
 *   idx_dev device, P ints, written
 *   cuda_stream  stream of the launch (NULL = legacy default stream)
 * Asynchronous.  The first call on each device looks up the array's device
 * address with that device current, so it should come before any stream
 * capture.  All calls share the array and it keeps the previous call's
 * contents (the first P entries are overwritten before use); calls whose
 * kernels may overlap on the GPU race and must be serialised by the caller.
 * Returns BP_ERR_INVALID_ARG for NULL pointers or out-of-range arguments,
 * BP_ERR_CUDA if the device address lookup or the launch fails, or if a CUDA
 * error was already pending on entry (nothing is launched then, and the
 * pending error is left in place for its owner). */
enum { BP_NOALLOC_MAX_P = 1 << 20 };
bp_status bp_resample_noalloc(const double* w_dev, int P, uint64_t seed, int n, int kind, int index,
                              int* idx_dev, void* cuda_stream);

/* ------------------------------------------------------------------ PCRLB
 * Posterior Cramer-Rao lower bounds (Sec. VI, Supplementary Sec. S-VII) as accuracy
 * references.  Global parameters: the MT state (6), the K SFV positions (3K), the
 * nuisance phases (coherent = 1: one per component shared by all PAs, K+1; 0: one per
 * component and PA, (K+1) J), the moduli ((K+1) J) and the common noise variance: dim =
 * 6 + 3K + nph + (K+1) J + 1, components with the LoS first.  For the bound the complex
 * amplitudes rho~ include path loss and carrier phase, and the array response is
 * unit-modulus (Sec. S-VII).  Reading: the SFV rows of the Jacobian are the full
 * derivative of the PA-to-virtual-MT vector (the printed mapping block holds the
 * reflection fixed).  FP64, synchronous; 0 <= K <= 15. */

/* Bayesian snapshot FIM: the mean over M realisations of sum_j G_j J_ch^(j) G_j^T
 * (eq. FIMclassic; Table S-I for J_ch).  x: M x 6 MT states, sfv: M x K x 3, rho:
 * M x J x (K+1) complex (interleaved) amplitudes rho~, eta: noise variance; fim: dim x
 * dim, written.  Host pointers.  BP_ERR_CAPACITY if the shape exceeds shared memory. */
bp_status bp_pcrlb_fim(const bp_geometry* geom, int K, int coherent, int M, const double* x, const double* sfv,
                       const double* rho, double eta, double* fim, void* cuda_stream);

/* The recursion J_{n|n} = J_B,n + (F J_{n-1|n-1}^-1 F^T + Q)^-1 (eq. posteriorCRLB,
 * priorFIM) from J_{1|0} = J10 over N steps of snapshot FIMs Jsnap (N x dim x dim), with
 * PEB_n = sqrt(tr P[0:3, 0:3]) and MEB_{k,n} = sqrt(tr P over SFV k), P = J_{n|n}^-1
 * (peb: N, meb: N x K, written).  F, Q, J10: dim x dim.  Host pointers.  BP_ERR_NUMERIC
 * if an inverted matrix is not positive definite. */
bp_status bp_pcrlb_recursion(int dim, int N, int K, const double* F, const double* Q, const double* J10,
                             const double* Jsnap, double* peb, double* meb, void* cuda_stream);

/* ------------------------------------------------------------------ batches
 * Many independent filters ("scenarios": each its own geometry, parameters,
 * particle count and PF capacity) stepped together on one GPU.  The paper has
 * no counterpart; each scenario runs exactly the step of bp_predict +
 * bp_update (Sec. IV), so its results are those of a single handle created
 * with the same arguments.
 *
 * Execution: the scenarios are ordered by their estimated cost (largest
 * first) and dealt over n_streams CUDA streams, each stream taking the next
 * scenario when its queue is the shortest (longest-processing-time list
 * scheduling); the GPU runs the streams' kernels concurrently.  Scenarios on
 * one stream run one after another, so with shared_workspace = 1 they share
 * one per-step workspace (geometry records, bases, likelihoods, CDFs), sized
 * for the largest of them; only the particle state stays per scenario.  With
 * use_graph = 1 and every scenario's PF count fixed (Q = 0 and T_pru = 0), the
 * whole batch step is captured once into a CUDA graph per particle-buffer
 * parity and replayed (no per-launch host cost); otherwise the launches are
 * issued directly and, where a PF count can change, the batch step ends with
 * one synchronisation that reads back every scenario's count.
 *
 * Diagnostics (bp_get_diag) of a scenario are unavailable with
 * shared_workspace = 1 (BP_ERR_STATE).  bp_batch_handle gives a scenario's
 * handle for bp_estimate, bp_get_state / bp_set_state and the other
 * single-handle calls (not bp_predict / bp_update / bp_free while the batch
 * exists); such calls on a handle synchronise its stream only. */
typedef struct bp_batch bp_batch;

typedef struct {
    const bp_geometry* geom;
    const bp_params* params;
    int P;             /* particles per belief */
    int S_max;         /* PF capacity (<= 64) */
    int S0;            /* PFs at time 0: the LoS and S0 - 1 drawn from the birth density
                          over the whole birth box (existence p_B, PR existence p_B^PR);
                          1 <= S0 <= S_max (bp_init uses 1) */
    uint64_t seed;     /* Philox key of the scenario */
} bp_scenario;

typedef struct {
    int n_streams;         /* 1..128 concurrent streams; 0 = 32 */
    int shared_workspace;  /* 1: one workspace per stream; 0: one per scenario */
    int use_graph;         /* 1: capture and replay the batch step where allowed */
    void* cuda_stream;     /* cudaStream_t every batch step is ordered after and before
                              (fork and join point); NULL = a blocking stream the batch
                              creates (ordered with the legacy default stream) */
} bp_batch_opts;

/* Creates the scenarios' handles (the time-0 beliefs of bp_init), the streams
 * and the workspaces.  opts may be NULL (32 streams, shared workspaces,
 * graphs on).  Synchronous.  On failure nothing is kept, *out is NULL and
 * bp_batch_last_error(NULL) gives the reason. */
bp_status bp_batch_init(const bp_scenario* sc, int n, const bp_batch_opts* opts, bp_batch** out);

/* One step (prediction and update) of every scenario.  z_dev: device pointer
 * to the scenarios' observations, concatenated in scenario order; scenario i
 * reads J_i x Nz_i complex FP32 values from element offset bp_batch_z_offset
 * (in floats).  Asynchronous unless a PF count can change (see above).  A
 * graph captured with one z_dev is re-captured when another pointer is
 * passed. */
bp_status bp_batch_step(bp_batch* b, const float* z_dev);

/* Float offset of scenario i's observations in z_dev, and the total floats. */
size_t bp_batch_z_offset(const bp_batch* b, int i);
size_t bp_batch_z_floats(const bp_batch* b);

/* Waits for every stream of the batch.  Returns BP_ERR_CUDA on a device error. */
bp_status bp_batch_sync(bp_batch* b);

/* Handle of scenario i (owned by the batch). */
bp_status bp_batch_handle(bp_batch* b, int i, bp_handle** h);

/* bp_set_tiles on scenario i; the captured step graphs are dropped and
 * captured again at the next bp_batch_step. */
bp_status bp_batch_set_tiles(bp_batch* b, int i, const bp_tiles* t);

/* Stream index a scenario was dealt to, and the bytes of device memory the
 * batch holds (state + workspaces), for inspection. */
int bp_batch_stream_of(const bp_batch* b, int i);
size_t bp_batch_device_bytes(const bp_batch* b);

/* Frees every scenario, stream, workspace and graph.  Synchronous. */
bp_status bp_batch_free(bp_batch* b);

/* Text of the last error on b (of the last bp_batch_init failure if b is NULL). */
const char* bp_batch_last_error(const bp_batch* b);

/* ------------------------------------------------------------------ proposal network
 * The network of the learned MT proposal (no counterpart in the paper, whose
 * proposal is the state-transition PDF): a perceptron 16 -> 64 -> 64 -> 16 with ReLU
 * after both hidden layers, BF16 weights, inputs and activations, FP32 accumulation on
 * the tensor cores.  Outputs y[0:3] = mean and y[3:6] = log standard deviation of a
 * Gaussian over a 3-vector (the remaining 10 outputs are unused); training minimises
 * the mean Gaussian negative log-likelihood of targets t (B x 3):
 *   L = (1/B) sum_i sum_a [ (t_ia - y_ia)^2 exp(-2 y_i,3+a) / 2 + y_i,3+a ].
 * Parameters (FP32 master copy, BP_MLP_NPARAM floats, in this order): W1 (64 x 16,
 * row = output unit), b1 (64), W2 (64 x 64), b2 (64), W3 (16 x 64), b3 (16).
 * The handle owns its parameters and Adam moments (beta1 0.9, beta2 0.999, eps 1e-8);
 * X (B x 16), T (B x 3), Y (B x 16) are FP32 device arrays, row-major.  Calls run on
 * the handle's stream.  Errors: BP_ERR_INVALID_ARG for NULL or out-of-range
 * arguments, BP_ERR_CUDA for allocation or launch failures, BP_ERR_TIMEOUT when a
 * bounded tensor-core wait gave up (results invalid). */
enum { BP_MLP_IN = 16, BP_MLP_HIDDEN = 64, BP_MLP_OUT = 16, BP_MLP_NPARAM = 6288 };
typedef struct bp_mlp bp_mlp;

/* Copies the initial parameters (host, BP_MLP_NPARAM floats) to the device; Adam
 * moments start at zero.  Synchronous. */
bp_status bp_mlp_create(const float* params_host, void* cuda_stream, bp_mlp** out);

/* The current parameters to host memory.  Synchronous. */
bp_status bp_mlp_get_params(bp_mlp* h, float* params_host);

/* Y = network(X) for B rows.  Synchronous (checks the tensor-core status). */
bp_status bp_mlp_forward(bp_mlp* h, const float* X_dev, int B, float* Y_dev);

/* Gradient of L with respect to every parameter (grad_dev: BP_MLP_NPARAM floats,
 * device) and B L (loss_dev: one float, device, may be NULL), parameters unchanged.
 * Synchronous. */
bp_status bp_mlp_grads(bp_mlp* h, const float* X_dev, const float* T_dev, int B, float* grad_dev, float* loss_dev);

/* One Adam step with learning rate lr on the gradient of L over this batch; loss_dev
 * (device, may be NULL) receives B L before the step.  Asynchronous: bp_mlp_sync
 * waits and reports a tensor-core timeout of any step since the last check. */
bp_status bp_mlp_train_step(bp_mlp* h, const float* X_dev, const float* T_dev, int B, float lr, float* loss_dev);
bp_status bp_mlp_sync(bp_mlp* h);

bp_status bp_mlp_free(bp_mlp* h);
const char* bp_mlp_last_error(const bp_mlp* h);

/* ------------------------------------------------------------------ learned MT proposal
 * Attaches a proposal network to a filter (NULL detaches; the caller keeps the network
 * alive while attached).  With a network attached, every bp_update first redraws the
 * NCV process noise of each MT particle from N(mu, diag s^2) in units of sigma_v, with
 * (mu, log s) = the network's outputs (log s clamped to [-4, 1]) for the input row
 *   [(F x_{n-1} - xbar)_pos / 0.01 m, (F x_{n-1} - xbar)_vel / 0.1 m/s,
 *    xbar_pos in ROI units (3), Re, Im of rho_j conj(rho_0) / |rho_0| for j = 1..3 (6), |rho_0|],
 * xbar the weighted mean of the predicted particles and rho_j the normalised correlation
 * psi_j(xbar)^H z_j / (|psi_j| |z_j|) of the LoS steering vector with z_j, and multiplies
 * each prediction weight by N(u; 0, I) / N(u; mu, s^2) before normalising them (the
 * importance ratio of the transition to the proposal, which keeps the posterior exact).
 * Random draws: Philox purpose 15.  At most 4 PAs; not on handles of a batch
 * (BP_ERR_STATE).  Diagnostics: BP_DIAG_LPROP. */
bp_status bp_set_mt_proposal(bp_handle* h, bp_mlp* net);

/* Training samples of the proposal network simulated from the model on the GPU (n rows
 * of X (n x 16) and targets T (n x 3), device FP32): a previous true state uniform in
 * the ROI of prm (velocity uniform within +-v_max), its NCV successor, a previous
 * posterior mean with errors N(0, err_pos^2) / N(0, err_vel^2) and a particle around it
 * with spreads spread_pos / spread_vel, the observation of the successor (LoS and the K
 * surfaces sfv (K x 3, host) with moduli rho_abs (K + 1, host, LoS first), uniform
 * phases common to all PAs (coherent = 1) or drawn per PA (coherent = 0), complex
 * Gaussian noise of variance eta), the input row at the
 * predicted mean as above, and the target u that carries the particle's F x_{n-1} to the
 * true successor (least squares through Gamma).  0 <= K <= 64, J <= 4.  Synchronous. */
bp_status bp_lp_dataset(const bp_geometry* geom, const bp_params* prm, int K, const double* sfv, const double* rho_abs,
                        double eta, int coherent, double err_pos, double err_vel, double spread_pos, double spread_vel, int n,
                        uint64_t seed, float* X_dev, float* T_dev, void* cuda_stream);

#ifdef __cplusplus
}
#endif
#endif /* BP_H */
