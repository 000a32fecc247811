// Internal definitions of libbp: device constants, RNG, geometry and small
// numeric helpers shared by the kernels.  sm_103a only.
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>
#include <math.h>

#include "../../include/bp.h"

namespace bp {

constexpr int J_MAX = 16;
constexpr int NF_MAX = 128;
constexpr int MY_MAX = 16;
constexpr int MZ_MAX = 16;
constexpr int NZ_MAX = 2048;
constexpr int S_CAP_MAX = 64;

// Geometry and parameters, passed to kernels by value (constant bank).
struct DevGeom {
    int J, Nf, My, Mz, Nz;
    double fc, c, lam, B;
    double p_pa[J_MAX][3];
    double R[J_MAX][9];      // row-major, columns = local axes (global coords)
    double f[NF_MAX];        // baseband frequencies
    double py[MY_MAX], pz[MZ_MAX];
    // float-float constants for phases in cycles: 1/lambda, f_k/c; FP32 p/lambda
    float inv_lam_hi, inv_lam_lo;
    float fc_hi[NF_MAX], fc_lo[NF_MAX];
    float py_l[MY_MAX], pz_l[MZ_MAX];     // p_y / lambda, p_z / lambda (float-float with *_lo)
    float py_lo[MY_MAX], pz_lo[MZ_MAX];
    float amp_c;             // lambda / (4 pi)
    // the PA positions and rotations as FP32 pairs (hi + lo), for the float-float geometry
    float pa_h[J_MAX][3], pa_l[J_MAX][3];
    float R_h[J_MAX][9], R_l[J_MAX][9];
};

struct DevParams {
    double T, sigma_v;
    int motion_dims;
    double c_eta, c_gamma, sigma_mu, sigma_sfv;
    double pS, pS_pr, pR_pr, pB_pr, mu_B, pB;   // pB = birth probability per partition
    int Q;
    double T_dec, T_pru, gamma_max, mu_max, eta_min, eta_max;
    double p_min[3], p_max[3], v_max[3];
    int zero_mean, mvec_scaling, regularize;
    int birth_proposal, N_g;
    uint32_t key0, key1;
    int P, S_max;
};

// ------------------------------------------------------------------ Philox4x32-10
// Salmon, Moraes, Dror, Shaw (SC'11): 10 rounds, multipliers 0xD2511F53 and
// 0xCD9E8D57, Weyl increments 0x9E3779B9 and 0xBB67AE85.
struct U4 { uint32_t x, y, z, w; };

__host__ __device__ inline U4 philox(uint32_t c0, uint32_t c1, uint32_t c2, uint32_t c3, uint32_t k0, uint32_t k1) {
    #pragma unroll
    for (int r = 0; r < 10; ++r) {
        const uint64_t p0 = (uint64_t)0xD2511F53u * c0;
        const uint64_t p1 = (uint64_t)0xCD9E8D57u * c2;
        const uint32_t hi0 = (uint32_t)(p0 >> 32), lo0 = (uint32_t)p0;
        const uint32_t hi1 = (uint32_t)(p1 >> 32), lo1 = (uint32_t)p1;
        const uint32_t n0 = hi1 ^ c1 ^ k0, n2 = hi0 ^ c3 ^ k1;
        c0 = n0; c1 = lo1; c2 = n2; c3 = lo0;
        k0 += 0x9E3779B9u; k1 += 0xBB67AE85u;
    }
    return U4{c0, c1, c2, c3};
}

// draw purposes (bits 31..16 of the third counter word); must match the oracle
enum : uint32_t {
    RNG_MT_PREDICT = 1, RNG_ETA_PREDICT = 2, RNG_PF_GAUSS = 3, RNG_PF_GAMMA = 4, RNG_BIRTH = 5,
    RNG_RESAMPLE = 6, RNG_JITTER_MT = 7, RNG_JITTER_PF = 8, RNG_JITTER_ETA = 9, RNG_INIT_MT = 10,
    RNG_INIT_ETA = 11, RNG_SYNTH_NOISE = 12, RNG_BIRTH_CAND = 13, RNG_BIRTH_PROP = 14,
    RNG_LEARNED_PROP = 15, RNG_LP_DATA = 16
};
constexpr int MAX_GAMMA_ATTEMPTS = 16;
// Range check of a data-dependent index (checked builds, -DBP_CHECKED): a failed check
// raises bit 2 of the kernel error word, which bp_estimate reports, and the caller skips
// the access.  In normal builds the check compiles away.
constexpr int KERR_TIMEOUT = 1, KERR_INDEX = 2;
__device__ __forceinline__ bool bp_in_range(long long i, long long n, int* kerr) {
#ifdef BP_CHECKED
    if (i < 0 || i >= n) {
        atomicOr(kerr, KERR_INDEX);
        return false;
    }
#else
    (void)i; (void)n; (void)kerr;
#endif
    return true;
}

// estimate status: the observation of the last update held NaN or Inf (reported as
// BP_ERR_NUMERIC with its own message)
constexpr int EST_STATUS_BAD_Z = 100;

__device__ inline U4 draw(const DevParams& P, uint32_t item, uint32_t n, uint32_t purpose, uint32_t sub, uint32_t block) {
    return philox(item, n, (purpose << 16) | (sub & 0xFFFFu), block, P.key0, P.key1);
}

// ((x >> 8) + 1/2) 2^-24: uniform in (0,1), exact in FP32
__device__ inline float u24(uint32_t x) { return ((float)(x >> 8) + 0.5f) * 5.9604644775390625e-8f; }
// the same uniform exactly, ((x >> 8) + 1/2) 2^-24 in FP64 (the FP32 form above rounds the
// half away for x >= 2^31: within FP32 rounding of the draws it feeds)
__device__ inline double u24d(uint32_t x) { return ((double)(x >> 8) + 0.5) * 5.9604644775390625e-8; }
// (x + 1/2) 2^-32: uniform in (0,1), exact in FP64
__host__ __device__ inline double u32d(uint32_t x) { return ((double)x + 0.5) * 2.3283064365386963e-10; }

// -2 log u for the 24-bit uniform u = ((x >> 8) + 1/2) 2^-24, to FP32 accuracy: for u >= 1/2,
// log u = log1p(-(1 - u)) with 1 - u formed exactly from the integer complement (u itself
// rounds in FP32 there, which near 1 would put large relative errors on small radii)
__device__ inline float neg2log_u24(uint32_t x) {
    const uint32_t k = x >> 8;
    if (k >= (1u << 23)) {
        const float om = ((float)((1u << 24) - 1u - k) + 0.5f) * 5.9604644775390625e-8f;
        return -2.0f * log1pf(-om);
    }
    return -2.0f * logf(((float)k + 0.5f) * 5.9604644775390625e-8f);
}

// 2u for the same uniform as an exact FP32 argument of sincospi: for u >= 1/2 the
// equivalent angle 2u - 2 = -2 (1 - u) (a whole turn removed), 1 - u from the complement
__device__ inline float twice_u24_turn(uint32_t x) {
    const uint32_t k = x >> 8;
    if (k >= (1u << 23)) return -2.0f * (((float)((1u << 24) - 1u - k) + 0.5f) * 5.9604644775390625e-8f);
    return 2.0f * (((float)k + 0.5f) * 5.9604644775390625e-8f);
}

// Box-Muller pair in FP32 from two 24-bit uniforms (radius and angle from exact arguments)
__device__ inline void box_muller_f(uint32_t a, uint32_t b, float& n0, float& n1) {
    const float r = sqrtf(neg2log_u24(a));
    float s, c;
    sincospif(twice_u24_turn(b), &s, &c);
    n0 = r * c;
    n1 = r * s;
}

// `count` (<= 8) standard normals for one item, blocks 0, 1 in order
__device__ inline void normals8(const DevParams& P, uint32_t item, uint32_t n, uint32_t purpose, uint32_t sub,
                                int count, float* out) {
    for (int blk = 0; blk * 4 < count; ++blk) {
        const U4 r = draw(P, item, n, purpose, sub, blk);
        float a0, a1, b0, b1;
        box_muller_f(r.x, r.y, a0, a1);
        box_muller_f(r.z, r.w, b0, b1);
        const float v[4] = {a0, a1, b0, b1};
        for (int i = 0; i < 4 && blk * 4 + i < count; ++i) out[blk * 4 + i] = v[i];
    }
}

// Marsaglia & Tsang (2000) Gamma(shape >= 1, scale) in FP64; attempt a uses block a
__device__ inline double gamma_draw(const DevParams& P, uint32_t item, uint32_t n, uint32_t purpose, uint32_t sub,
                                    double shape, double scale) {
    const double d = shape - 1.0 / 3.0;
    const double c = 1.0 / sqrt(9.0 * d);
    for (int a = 0; a < MAX_GAMMA_ATTEMPTS; ++a) {
        const U4 r = draw(P, item, n, purpose, sub, (uint32_t)a);
        const double g = sqrt(-2.0 * log(u32d(r.x))) * cospi(2.0 * u32d(r.y));
        const double t = 1.0 + c * g;
        const double v = t * t * t;
        if (v <= 0.0) continue;
        const double u = u32d(r.z);
        if (log(u) < 0.5 * g * g + d - d * v + d * log(v)) return d * v * scale;
    }
    return shape * scale;
}

// ------------------------------------------------------------------ geometry (FP64)
// Local PA -> VM vector r' = R^T H (p - p_va) (eq. rangep, house, posPA-SB);
// returns |r'| and the local unit vector.
struct PathGeo { double d, ux, uy, uz; };

__device__ inline PathGeo path_geo(const DevGeom& G, int j, double px, double py, double pz,
                                   double sx, double sy, double sz, bool los) {
    double rx, ry, rz;
    const double ax = G.p_pa[j][0], ay = G.p_pa[j][1], az = G.p_pa[j][2];
    if (los) {
        rx = px - ax; ry = py - ay; rz = pz - az;
    } else {
        const double nn = sx * sx + sy * sy + sz * sz;
        const double coef = 2.0 * (ax * sx + ay * sy + az * sz) / nn - 1.0;
        const double vx = ax - coef * sx, vy = ay - coef * sy, vz = az - coef * sz;
        const double qx = px - vx, qy = py - vy, qz = pz - vz;
        const double t = 2.0 * (sx * qx + sy * qy + sz * qz) / nn;
        rx = qx - t * sx; ry = qy - t * sy; rz = qz - t * sz;
    }
    const double* R = G.R[j];
    const double lx = R[0] * rx + R[3] * ry + R[6] * rz;
    const double ly = R[1] * rx + R[4] * ry + R[7] * rz;
    const double lz = R[2] * rx + R[5] * ry + R[8] * rz;
    const double d = sqrt(lx * lx + ly * ly + lz * lz);
    const double inv = 1.0 / d;
    return PathGeo{d, lx * inv, ly * inv, lz * inv};
}

// cis(2 pi t) for a phase in cycles, reduced to its fractional part first
__device__ inline double2 cis_cycles(double t) {
    const double f = t - rint(t);
    double s, c;
    sincospi(2.0 * f, &s, &c);
    return make_double2(c, s);
}

// element (f, y, m) of psi_j in FP64: lambda/(4 pi d) exp(j 2 pi (-(fc + f_f) d / c +
// (p_y uy + p_z uz) / lambda))
__device__ inline double2 steer_elem(const DevGeom& G, const PathGeo& g, int f, int y, int m) {
    const double amp = G.lam / (4.0 * M_PI * g.d);
    const double cyc = -(G.fc + G.f[f]) * g.d / G.c + (G.py[y] * g.uy + G.pz[m] * g.uz) / G.lam;
    const double2 e = cis_cycles(cyc);
    return make_double2(amp * e.x, amp * e.y);
}

// fractional part in [-1/2, 1/2]
__device__ inline double frac_c(double t) { return t - rint(t); }

// Fractional part (in [-1/2, 1/2]) of the float-float product (ah + al)(bh + bl),
// with the leading product split exactly by FMA (Dekker/Ogita two-product):
// about 1e-8 absolute accuracy for products up to ~1e3 cycles, all in FP32.
__device__ inline float ff_frac_mul(float ah, float al, float bh, float bl) {
    const float p = ah * bh;
    const float e = fmaf(ah, bh, -p);
    const float n = rintf(p);
    const float t = e + ah * bl + al * bh;
    return (p - n) + t;
}

// The same fraction as an unevaluated pair hi + lo (hi = p - rint(p) exactly, lo the
// low-order terms), for a phase kept beyond FP32 rounding.
__device__ inline void ff_frac_mul2(float ah, float al, float bh, float bl, float& hi, float& lo) {
    const float p = __fmul_rn(ah, bh);
    const float e = fmaf(ah, bh, -p);
    hi = __fsub_rn(p, rintf(p));
    lo = fmaf(ah, bl, fmaf(al, bh, e));
}
// (cos, sin) of pi (a + b) for |b| < 1e-4: sincospi of the leading part and the
// first-order term of the small one (second order below 5e-8 relative)
__device__ inline float2 cispi_ff(float a, float b) {
    float sn, cs;
    sincospif(a, &sn, &cs);
    const float pb = 3.14159265358979f * b;
    return make_float2(fmaf(-pb, sn, cs), fmaf(pb, cs, sn));
}

// Geometry record of one (particle, feature, PA): distance |r'| as a float-float
// pair and the local direction cosines u_y, u_z (float-float, low parts apart).
struct GeoRec { float d_hi, d_lo, uy, uz; };

// ------------------------------------------------------------------ complex / double-float helpers
__host__ __device__ inline float2 cmul(float2 a, float2 b) { return make_float2(a.x * b.x - a.y * b.y, a.x * b.y + a.y * b.x); }
__host__ __device__ inline float2 cmulc(float2 a, float2 b) {  // conj(a) * b
    return make_float2(a.x * b.x + a.y * b.y, a.x * b.y - a.y * b.x);
}
__host__ __device__ inline double2 zmul(double2 a, double2 b) { return make_double2(a.x * b.x - a.y * b.y, a.x * b.y + a.y * b.x); }
__host__ __device__ inline double2 zmulc(double2 a, double2 b) { return make_double2(a.x * b.x + a.y * b.y, a.x * b.y - a.y * b.x); }

// ------------------------------------------------------------------ float-float (FP32 pairs)
// Error-free transformations (Knuth TwoSum, Dekker/FMA TwoProd) and the
// float-float operations built on them (about 44 significant bits).
__device__ inline void two_sum(float a, float b, float& s, float& e) {
    s = __fadd_rn(a, b);
    const float bb = __fsub_rn(s, a);
    e = __fadd_rn(__fsub_rn(a, __fsub_rn(s, bb)), __fsub_rn(b, bb));
}
__device__ inline void fast_two_sum(float a, float b, float& s, float& e) {   // |a| >= |b|
    s = __fadd_rn(a, b);
    e = __fsub_rn(b, __fsub_rn(s, a));
}
struct ff { float hi, lo; };
__device__ inline ff ff_add(ff x, ff y) {
    float s, e;
    two_sum(x.hi, y.hi, s, e);
    e = __fadd_rn(e, __fadd_rn(x.lo, y.lo));
    ff r;
    fast_two_sum(s, e, r.hi, r.lo);
    return r;
}
__device__ inline ff ff_neg(ff x) { return ff{-x.hi, -x.lo}; }
__device__ inline ff ff_mul(ff x, ff y) {
    const float p = __fmul_rn(x.hi, y.hi);
    float e = fmaf(x.hi, y.hi, -p);
    e = fmaf(x.hi, y.lo, fmaf(x.lo, y.hi, e));
    ff r;
    fast_two_sum(p, e, r.hi, r.lo);
    return r;
}
__device__ inline ff ff_prod(float a, float b) {       // exact product of two floats
    const float p = __fmul_rn(a, b);
    return ff{p, fmaf(a, b, -p)};
}
__device__ inline ff ff_div(ff x, ff y) {              // one Newton correction
    const float q = __fdiv_rn(x.hi, y.hi);
    const ff r = ff_add(x, ff_neg(ff_mul(ff{q, 0.f}, y)));
    const float q2 = __fdiv_rn(r.hi, y.hi);
    ff out;
    fast_two_sum(q, q2, out.hi, out.lo);
    return out;
}
struct cff { ff re, im; };
__device__ inline cff cff_add(cff a, cff b) { return cff{ff_add(a.re, b.re), ff_add(a.im, b.im)}; }
__device__ inline cff cff_sub(cff a, cff b) { return cff{ff_add(a.re, ff_neg(b.re)), ff_add(a.im, ff_neg(b.im))}; }
__device__ inline cff cff_mul(cff a, cff b) {
    return cff{ff_add(ff_mul(a.re, b.re), ff_neg(ff_mul(a.im, b.im))), ff_add(ff_mul(a.re, b.im), ff_mul(a.im, b.re))};
}
__device__ inline cff cff_mulc(cff a, cff b) {         // conj(a) * b
    return cff{ff_add(ff_mul(a.re, b.re), ff_mul(a.im, b.im)), ff_add(ff_mul(a.re, b.im), ff_neg(ff_mul(a.im, b.re)))};
}
__device__ inline cff cff_from(float2 v) { return cff{ff{v.x, 0.f}, ff{v.y, 0.f}}; }
// exact conj(a) * b of two FP32 complex numbers
__device__ inline cff cff_prodc(float2 a, float2 b) {
    return cff{ff_add(ff_prod(a.x, b.x), ff_prod(a.y, b.y)), ff_add(ff_prod(a.x, b.y), ff_neg(ff_prod(a.y, b.x)))};
}

// acc += |v|^2 with exact squares; acc.lo is left unnormalised
__device__ inline void ff_acc_sq(ff& acc, float2 v) {
    const float p1 = __fmul_rn(v.x, v.x), e1 = fmaf(v.x, v.x, -p1);
    const float p2 = __fmul_rn(v.y, v.y), e2 = fmaf(v.y, v.y, -p2);
    float s, e, t;
    two_sum(acc.hi, p1, s, e);
    two_sum(s, p2, acc.hi, t);
    acc.lo = __fadd_rn(acc.lo, __fadd_rn(__fadd_rn(e, t), __fadd_rn(e1, e2)));
}
__device__ inline double ff_to_d(ff v) { return (double)v.hi + (double)v.lo; }
// running product of positive factors as a float-float mantissa in [0.5, 1) and an exponent
struct ffexp { ff m; int e; };
__device__ inline void ffexp_mul(ffexp& x, ff f) {
    x.m = ff_mul(x.m, f);
    int e;
    frexpf(x.m.hi, &e);
    x.m.hi = ldexpf(x.m.hi, -e);
    x.m.lo = ldexpf(x.m.lo, -e);
    x.e += e;
}
// log of the product: logf is applied to the mantissa only (|log m| < 0.7, so its
// 1-ulp error is below 1e-7), the exponent enters exactly
__device__ inline double ffexp_log(const ffexp& x) {
    return (double)logf(x.m.hi) + (double)(x.m.lo / x.m.hi) + (double)x.e * 0.69314718055994530942;
}

__device__ inline double warp_sum_d(double v) {
    #pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    return v;
}
__device__ inline float warp_sum_f(float v) {
    #pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    return v;
}
__device__ inline ff warp_sum_ff(ff v) {
    #pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        const ff w{__shfl_xor_sync(0xffffffffu, v.hi, o), __shfl_xor_sync(0xffffffffu, v.lo, o)};
        v = ff_add(v, w);
    }
    return v;
}
__device__ inline double warp_max_d(double v) {
    #pragma unroll
    for (int o = 16; o > 0; o >>= 1) v = fmax(v, __shfl_xor_sync(0xffffffffu, v, o));
    return v;
}

// ------------------------------------------------------------------ device state
// Pointers of one filter's device buffers (owned by the handle).
struct DevState {
    // particles, two buffers each (resampling writes the other one)
    float* x[2];      // 6 x P
    float* phi[2];    // S_max x 6 x P
    float* eta[2];    // J x P
    int cur;
    // weights (FP64)
    double* w_x;      // P      belief / w_beta
    double* w_y;      // S_max x P  belief weights
    double* w_alpha;  // S_max x P  PF prediction weights
    double* w_eta;    // J x P  belief / w_xi
    double* p_pr;     // S_max x J  belief p(r=1)
    double* zeta;     // S_max x J  zeta(1)
    double* p_s;      // S_max
    double* wn_x;     // P          normalised weights before resampling
    double* wn_y;     // S_max x P
    double* wn_eta;   // J x P
    // log weights / likelihoods of the current update
    double* lw_x;     // P
    double* lw_y;     // S_max x P   (Delta_kappa summed over j, without log w_alpha)
    double* lw_eta;   // J x P
    double* llr_w;    // S_max x J   log omega(1) - log omega(0)
    // message table (FP64) and derived per-(s,j) quantities
    float4* geo;      // [S_max][J][P] GeoRec of the current prediction: |r'| (hi, lo), u_y, u_z
    float2* geo_lo;   // [S_max][J][P] low parts of u_y, u_z
    int* flags;       // [0] count of flagged particles, then their indices (iota repair)
    float* iota_err;  // P   error bound (nats) of the FP32 log iota~ sum (k_iota_bulk)
    unsigned long long* iota_key;   // largest lower bound of the MT log-weights, as an ordered key
    double* tab;      // [4][S_max][J][Nz] double2 : m, mw, mu3, mu4
    double* tab_part; // table partial sums [nsplit][3][S_max][J][Nz] double2
    double* W;        // S_max    sum_p w_alpha
    double* eta_bar;  // J
    // kappa stage outputs (per (s,j))
    float2* kV;       // [S_max][J][Nz][S_cap]   whitened basis, column S_cap-1 = r0 (FP32 part)
    float2* kr0l;     // [S_max][J][Nz]          low part of r0 (r0 = FP32 part + low part)
    float2* kdl;      // [S_max][J][S_cap]       1/lambda_c of the eigen-whitened basis (.x; zero-padded)
    float* kB;        // TF32 B tiles of the tensor-core PF likelihood (or null): pass 1
                      // [S][J][rounds][hi, lo][2 S_cap x 32], then pass 2 [S][J][groups][S_cap/16][hi, lo][64 x 32]
    int* kerr;        // nonzero after a bounded wait of a kernel gave up (reported by bp_estimate)
    float2* ky0;      // [S_max][J][S_cap]       y~0 = V^H e0 / eta_bar (zero-padded)
    double* kJ0;      // [S_max][J]              |r0|^2/eta_bar
    // nu stage outputs (per j)
    double* nu_T;     // [J][S_max] diag a_k, [J][S_max] |offdiag|^2, [J][S_max] double2 b'
    double* nu_c;     // [J][2] |e|^2, constant
    // normalisation scratch
    double* red_part; // block partials
    double* bel;      // per-belief results (see k_norm.cu)
    float* Lchol;     // per-belief jitter factors
    int* idx;         // (1 + S_max + J) x P resampling indices
    int* ctrl;        // [0] S, [1] S_next, [2] births_skipped, [3] status, [4..] keep map
    int* step;        // [0] step index n of the Philox counters, advanced on the device (k_step_advance)
    double* bprop;    // birth proposal scratch, real part (BpropLayout), or null
    double2* bprop_c; // birth proposal scratch, complex part: steering matrices and residuals
    double* est;      // estimates buffer
};

}  // namespace bp
