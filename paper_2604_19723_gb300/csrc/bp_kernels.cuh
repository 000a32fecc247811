// Kernel launch wrappers and shared buffer layouts of libbp.
#pragma once
#include "bp_internal.cuh"

namespace bp {

// Scratch of the birth proposal (k_birth.cu).  Complex part (double2): the steering
// matrices Psi_j [J][S_max][Nz] and the residuals z~_j [J][Nz].  Real part (double): the
// estimates [1 + S_max][3] (MT first), per new PF q < Q the statistics [32] (valid, i*,
// sum of costs, mu [3], C [3][3], L [3][3]), the costs [Q][N_g], the candidates
// [Q][N_g][3], the proposal draws [Q][P][3] and per-block sums of their weights.
struct BpropLayout {
    int J, Nz, S_max, N_g, Q, P;
    __host__ __device__ size_t psi(int j) const { return (size_t)j * S_max * Nz; }
    __host__ __device__ size_t zres(int j) const { return (size_t)J * S_max * Nz + (size_t)j * Nz; }
    __host__ __device__ size_t c_total() const { return (size_t)J * S_max * Nz + (size_t)J * Nz; }
    __host__ __device__ size_t means() const { return 0; }
    __host__ __device__ size_t stats(int q) const { return 3 * (size_t)(1 + S_max) + 32 * (size_t)q; }
    __host__ __device__ size_t costs() const { return 3 * (size_t)(1 + S_max) + 32 * (size_t)Q; }
    __host__ __device__ size_t cand() const { return costs() + (size_t)Q * N_g; }
    __host__ __device__ size_t pos(int q) const { return cand() + (size_t)Q * N_g * 3 + (size_t)q * P * 3; }
    __host__ __device__ size_t parts(int q) const { return pos(Q) + (size_t)q * ((P + 255) / 256); }
    __host__ __device__ size_t r_total() const { return parts(Q); }
};
inline BpropLayout bprop_layout(const DevGeom& G, const DevParams& Pm) {
    return BpropLayout{G.J, G.Nz, Pm.S_max, Pm.N_g, Pm.Q, Pm.P};
}
// the birth proposal of the new PFs S_L .. S_new - 1 (no-op unless enabled); returns launches
int launch_birth_proposal(const DevGeom& G, const DevParams& Pm, const DevState& D, int S_L, int S_new,
                          const float* z, cudaStream_t st);

// Largest dynamic shared memory a block may opt in to on the current device.
int smem_optin();
// Raises a kernel's dynamic shared-memory limit to the opt-in maximum less its static
// shared memory (once per kernel), not to one launch's need: launches of one kernel
// with different sizes from several streams, or replayed from a captured graph, then
// never meet a limit set for a smaller launch.
void smem_allow_max(const void* kernel);


// per-belief result buffer (doubles); belief index b: 0 = MT, 1 + s = PF s, 1 + S_max + j = eta_j
constexpr int BEL_STRIDE = 16;   // per belief: [0] max, [1] lse, [2] logC, [3] sum w^2 factor, [4..9] mean, [10] active dims
inline __host__ __device__ int bel_count(int S_max, int J) { return 1 + S_max + J; }
#define BEL_PPR 0   /* offset of the updated PR existence table inside D.bel (S_max x J) */
inline __host__ __device__ size_t bel_ppr_size(int S_max, int J) { return (size_t)S_max * J; }
inline __host__ __device__ size_t bel_rec(int S_max, int J, int b) { return bel_ppr_size(S_max, J) + (size_t)b * BEL_STRIDE; }
inline __host__ __device__ size_t bel_total(int S_max, int J) { return bel_ppr_size(S_max, J) + (size_t)bel_count(S_max, J) * BEL_STRIDE; }

// estimate buffer layout (doubles)
struct EstLayout {
    int S_max, J;
    __host__ __device__ size_t n() const { return 0; }
    __host__ __device__ size_t S() const { return 1; }
    __host__ __device__ size_t S_next() const { return 2; }
    __host__ __device__ size_t skipped() const { return 3; }
    __host__ __device__ size_t status() const { return 4; }
    __host__ __device__ size_t repaired() const { return 5; }
    __host__ __device__ size_t x_hat() const { return 6; }
    __host__ __device__ size_t ess() const { return 12; }
    __host__ __device__ size_t eta_hat() const { return 13; }
    __host__ __device__ size_t p_s() const { return 13 + J; }
    __host__ __device__ size_t phi_hat() const { return 13 + J + S_max; }
    __host__ __device__ size_t p_pr() const { return 13 + J + 7 * S_max; }
    __host__ __device__ size_t p_any() const { return 13 + J + 7 * S_max + S_max * J; }
    __host__ __device__ size_t declared() const { return 13 + J + 8 * S_max + S_max * J; }
    __host__ __device__ size_t total() const { return 13 + J + 9 * S_max + S_max * J; }
};

constexpr int RED_W = 29;   // per-block partial sums: S0, S1[6], S2[21] (upper, row-major), sum w^2

// Steering-vector factors from a geometry record (g, gl), FP32 arithmetic:
// psi = c (b kron a_y kron a_z), c = lambda/(4 pi d) e^{-i 2 pi d/lambda},
// b_f = e^{-i 2 pi f_f d/c}, a_y = e^{i 2 pi p_y u_y/lambda}, a_z = e^{i 2 pi p_z u_z/lambda}
// (eq. array-response, unit-modulus-array-response).  Every phase is formed as a
// float-float number of cycles (distance and direction cosines carry low parts) and
// enters sincospi with its first-order low-part correction, so the factors are exact
// to a few FP32 ulps; their products then decide the accuracy of psi.
__device__ inline void array_factors(const DevGeom& G, float4 g, float2 gl, float2* ay, float2* az, int stride) {
    for (int y = 0; y < G.My; ++y) {   // 2 p_y u_y / lambda half-cycles
        const float p = __fmul_rn(G.py_l[y], g.z);
        const float e = fmaf(G.py_l[y], gl.x, fmaf(G.py_lo[y], g.z, fmaf(G.py_l[y], g.z, -p)));
        ay[y * stride] = cispi_ff(2.0f * p, 2.0f * e);
    }
    for (int m = 0; m < G.Mz; ++m) {
        const float p = __fmul_rn(G.pz_l[m], g.w);
        const float e = fmaf(G.pz_l[m], gl.y, fmaf(G.pz_lo[m], g.w, fmaf(G.pz_l[m], g.w, -p)));
        az[m * stride] = cispi_ff(2.0f * p, 2.0f * e);
    }
}
// the amplitude and carrier factor A e^{-i 2 pi d / lambda} of the steering vector
__device__ inline float2 carrier_factor(const DevGeom& G, float4 g) {
    const float d = g.x + g.y;
    const float A = G.amp_c / d;
    float h, l;
    ff_frac_mul2(g.x, g.y, G.inv_lam_hi, G.inv_lam_lo, h, l);
    const float2 c = cispi_ff(-2.0f * h, -2.0f * l);
    return make_float2(A * c.x, A * c.y);
}
// frequency factor b_f = e^{-i 2 pi d f_f / c}
__device__ inline float2 freq_factor(const DevGeom& G, float4 g, int f) {
    float h, l;
    ff_frac_mul2(g.x, g.y, G.fc_hi[f], G.fc_lo[f], h, l);
    return cispi_ff(-2.0f * h, -2.0f * l);
}
__device__ inline float2 factors_from_geo(const DevGeom& G, float4 g, float2 gl, float2* b, float2* ay, float2* az, int stride) {
    const float2 Fc = carrier_factor(G, g);
    for (int f = 0; f < G.Nf; ++f) b[f * stride] = freq_factor(G, g, f);
    array_factors(G, g, gl, ay, az, stride);
    return Fc;
}

// As factors_from_geo, with the carrier phase folded into the frequency factor:
// psi = A (b' kron a_y kron a_z), b'_f = e^{-i 2 pi d (1/lambda + f_f/c)}, A = lambda/(4 pi d),
// one sincospi per frequency on the summed cycle count.  Returns A.
__device__ inline float factors_from_geo_folded(const DevGeom& G, float4 g, float2 gl, float2* b, float2* ay, float2* az, int stride) {
    const float d = g.x + g.y;
    float h0, l0;
    ff_frac_mul2(g.x, g.y, G.inv_lam_hi, G.inv_lam_lo, h0, l0);
    for (int f = 0; f < G.Nf; ++f) {
        float hf, lf, h, e;
        ff_frac_mul2(g.x, g.y, G.fc_hi[f], G.fc_lo[f], hf, lf);
        two_sum(h0, hf, h, e);
        b[f * stride] = cispi_ff(-2.0f * h, -2.0f * (e + l0 + lf));
    }
    array_factors(G, g, gl, ay, az, stride);
    return G.amp_c / d;
}

// e^{i 2 pi t} for a phase t = th + tl in cycles, as an unevaluated pair hi + lo good to
// ~1e-9: the nearest 1/256 of a cycle from a table of FP64-rounded (hi, lo) values, turned
// by the remainder angle phi (|phi| <= pi/256) through the angle-addition formulas with
// cos phi - 1 and sin phi from their Taylor series (terms beyond phi^5 below 1e-14)
__device__ inline void cis_pair(const float4* tab, float th, float tl, float2& hi, float2& lo) {
    const float n = rintf(th * 256.0f);
    const float rem = __fadd_rn(__fsub_rn(th, n * 0.00390625f), tl);   // th - n/256 is exact
    const float4 T = tab[((int)n) & 255];                                // cos hi, cos lo, sin hi, sin lo
    const float ph = 6.28318530717958648f * rem;
    const float p2 = ph * ph;
    const float cm1 = p2 * fmaf(p2, 1.0f / 24.0f, -0.5f);
    const float sp = ph * fmaf(p2, fmaf(p2, 1.0f / 120.0f, -1.0f / 6.0f), 1.0f);
    const float cr = fmaf(T.x, cm1, fmaf(-T.z, sp, T.y));
    const float ci = fmaf(T.z, cm1, fmaf(T.x, sp, T.w));
    fast_two_sum(T.x, cr, hi.x, lo.x);   // |cr| <= |T.x| unless T.x == 0
    fast_two_sum(T.z, ci, hi.y, lo.y);
}
// the table: e^{i 2 pi n / 256}, n = 0..255, in FP64 and split into FP32 pairs
__device__ inline void cis_table_fill(float4* tab, int tid, int nthreads) {
    for (int n = tid; n < 256; n += nthreads) {
        double sn, cs;
        sincospi((double)n / 128.0, &sn, &cs);
        const float ch = (float)cs, sh = (float)sn;
        tab[n] = make_float4(ch, (float)(cs - (double)ch), sh, (float)(sn - (double)sh));
    }
}
// steering factors of factors_from_geo_folded as (hi, lo) pairs (same phases, evaluated by
// cis_pair; element i at index i * stride); returns the amplitude A = lambda / (4 pi d)
__device__ inline float factors_from_geo_pairs(const DevGeom& G, const float4* tab, float4 g, float2 gl, float2* fh,
                                               float2* fl, int stride = 1) {
    const float d = g.x + g.y;
    float h0, l0;
    ff_frac_mul2(g.x, g.y, G.inv_lam_hi, G.inv_lam_lo, h0, l0);
    for (int f = 0; f < G.Nf; ++f) {
        float hf, lf, h, e;
        ff_frac_mul2(g.x, g.y, G.fc_hi[f], G.fc_lo[f], hf, lf);
        two_sum(h0, hf, h, e);
        cis_pair(tab, -h, -(e + l0 + lf), fh[f * stride], fl[f * stride]);
    }
    for (int y = 0; y < G.My; ++y) {
        const float p = __fmul_rn(G.py_l[y], g.z);
        const float e = fmaf(G.py_l[y], gl.x, fmaf(G.py_lo[y], g.z, fmaf(G.py_l[y], g.z, -p)));
        cis_pair(tab, p, e, fh[(G.Nf + y) * stride], fl[(G.Nf + y) * stride]);
    }
    for (int m = 0; m < G.Mz; ++m) {
        const float p = __fmul_rn(G.pz_l[m], g.w);
        const float e = fmaf(G.pz_l[m], gl.y, fmaf(G.pz_lo[m], g.w, fmaf(G.pz_l[m], g.w, -p)));
        cis_pair(tab, p, e, fh[(G.Nf + G.My + m) * stride], fl[(G.Nf + G.My + m) * stride]);
    }
    return G.amp_c / d;
}
// the frequency factor b'_f of factors_from_geo_pairs alone, from the record's distance
// (dh + dl) and its carrier cycle count (h0 + l0, from ff_frac_mul2 with 1/lambda)
__device__ inline void bprime_pair(const DevGeom& G, const float4* tab, float dh, float dl, float h0, float l0, int f,
                                   float2& hi, float2& lo) {
    float hf, lf, h, e;
    ff_frac_mul2(dh, dl, G.fc_hi[f], G.fc_lo[f], hf, lf);
    two_sum(h0, hf, h, e);
    cis_pair(tab, -h, -(e + l0 + lf), hi, lo);
}

// (ah + al)(bh + bl) as hi + lo: exact products of the high parts, the rounding of their
// sum, and the first-order cross terms
__device__ inline float4 cpair_mul(float2 ah, float2 al, float2 bh, float2 bl) {
    const float p1 = __fmul_rn(ah.x, bh.x), e1 = fmaf(ah.x, bh.x, -p1);
    const float p2 = __fmul_rn(ah.y, bh.y), e2 = fmaf(ah.y, bh.y, -p2);
    const float p3 = __fmul_rn(ah.x, bh.y), e3 = fmaf(ah.x, bh.y, -p3);
    const float p4 = __fmul_rn(ah.y, bh.x), e4 = fmaf(ah.y, bh.x, -p4);
    float rh, rl, ih, il;
    two_sum(p1, -p2, rh, rl);
    two_sum(p3, p4, ih, il);
    rl += (e1 - e2) + fmaf(ah.x, bl.x, fmaf(al.x, bh.x, -fmaf(ah.y, bl.y, al.y * bh.y)));
    il += (e3 + e4) + fmaf(ah.x, bl.y, fmaf(al.x, bh.y, fmaf(ah.y, bl.x, al.y * bh.x)));
    return make_float4(rh, ih, rl, il);
}

void launch_geom(const DevGeom& G, const DevParams& Pm, const DevState& D, int S, cudaStream_t st);
void launch_iota_repair(const DevGeom& G, const DevParams& Pm, const DevState& D, int S, const float* z, cudaStream_t st);

void launch_init(const DevGeom& G, const DevParams& Pm, const DevState& D, int S0, cudaStream_t st);
int launch_predict(const DevGeom& G, const DevParams& Pm, const DevState& D, int S_old, int S_new, cudaStream_t st);
void launch_row_sums(const DevParams& Pm, const DevState& D, int S, int J, cudaStream_t st);
// chunk_req: particles per shared-memory chunk (16, 32, 64, 128; 0 = 64), halved to fit
void launch_table(const DevGeom& G, const DevParams& Pm, const DevState& D, int S, int nsplit, int chunk_req,
                  cudaStream_t st);
// the PF basis stage; with a side stream the noise-likelihood tridiagonalisation runs there
// (forked after the Gram through ev_fork, ev_join recorded after it)
void launch_stage(const DevGeom& G, const DevParams& Pm, const DevState& D, int S, int SC, const float* z,
                  double* gram, double* nu_b, double* V64, cudaStream_t st, cudaStream_t side = nullptr,
                  cudaEvent_t ev_fork = nullptr, cudaEvent_t ev_join = nullptr);
// the PF-likelihood launch chosen from S, the shape and the tile requests (0 = built-in):
// column bucket sc, tensor-core kernel or CUDA-core one with mb blocks per SM and fch
// frequencies staged per chunk (smem bytes)
struct KappaPlan { int sc, mb, fch; bool tc; size_t smem; };
KappaPlan plan_kappa(const DevGeom& G, const DevState& D, int S, int SCA, int t_sc, int t_mb, int t_fch, int t_tc);
void launch_kappa(const DevGeom& G, const DevParams& Pm, const DevState& D, int S, int SCA, const KappaPlan& k,
                  cudaStream_t st);
bool kappa_tc_ok(const DevGeom& G, int SCA);
size_t kappa_btile_floats(const DevGeom& G, int S_max, int SCA);
// operand tiles of both tensor-core passes of the PF likelihood; returns launches
int launch_kappa_btile(const DevGeom& G, const DevState& D, int S, int SCA, cudaStream_t st);
// MT likelihood of every particle (returns its launches): the FP32 warp kernel with
// ratio flags below IOTA_FF_ALL_S PFs, else k_iota_bulk and the selection of the particles
// whose weights need the float-float evaluation; launch_iota_repair then evaluates the
// flagged particles in float-float
int launch_iota(const DevGeom& G, const DevParams& Pm, const DevState& D, int S, const float* z, cudaStream_t st);
int launch_iota_bulk(const DevGeom& G, const DevParams& Pm, const DevState& D, int S, const float* z, cudaStream_t st);
size_t iota_bulk_smem_bytes(const DevGeom& G, int S);
size_t iota_blk_smem_bytes(const DevGeom& G, int S);
void launch_nu(const DevGeom& G, const DevParams& Pm, const DevState& D, int S, cudaStream_t st);
int launch_normalize(const DevGeom& G, const DevParams& Pm, const DevState& D, int S, cudaStream_t st);
void launch_resample(const DevGeom& G, const DevParams& Pm, const DevState& D, int S, double* cdf, cudaStream_t st);
void launch_synth(const DevGeom& G, int n_steps, int step0, const double* x_pos, int K, const double* sfv,
                  const double* rho, const int* c_off, const double* c_sfv, const double* c_rho,
                  double* zbuf, uint32_t k0, uint32_t k1, cudaStream_t st);
void launch_synth_noise(const DevGeom& G, int n_steps, int step0, const double* zbuf, double eta, uint32_t k0,
                        uint32_t k1, float* z_out, cudaStream_t st);
void launch_power(const DevGeom& G, const double* zbuf, double* out, cudaStream_t st);

}  // namespace bp
