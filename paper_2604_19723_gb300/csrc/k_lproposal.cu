// Learned MT proposal (an extension; the paper draws MT particles from the NCV
// state-transition PDF).  At the start of an update, with the observation at hand,
// the NCV process noise of every MT particle is redrawn from a Gaussian whose mean and
// standard deviation the proposal network (k_mlp.cu) computes from the particle and a
// summary of z; the prediction weights take the importance ratio of the transition
// density to the proposal density, so the posterior the update computes is unchanged
// in expectation (exact as P grows) and only the particle placement differs.
//
// In units of the standard normal u of x_n = F x_{n-1} + Gamma sigma_v u:
//   inputs   X_p = [(F x_{n-1}^p - xbar)_pos / 0.01 m, (.)_vel / 0.1 m/s, s(z, xbar) (10)],
//            xbar the weighted mean of the predicted particles, s the shared summary
//            (xbar in ROI units (3); for PAs j = 1..3 the LoS correlation
//            rho_j = psi_j(xbar)^H z_j / (|psi_j| |z_j|) relative to PA 0 as
//            Re, Im of rho_j conj(rho_0) / |rho_0| (6); |rho_0| (1));
//   outputs  mu = y[0:3], log s = clamp(y[3:6], -4, 1);
//   draw     u = mu + s g, g ~ N(0, I) (Philox purpose 15, item p);
//   weight   w_beta^p <- w_beta^p N(u; 0, I) / N(u; mu, s^2) = w_beta^p exp(-|u|^2/2 + |g|^2/2 + sum log s),
//            then normalised; planar motion leaves z and v_z alone.
// F x_{n-1} is recovered from the predicted particle as x_n - Gamma sigma_v u_prior with
// the prediction's own draws (Philox purpose 1), recomputed.
//
// k_lp_dataset simulates training samples from the model: previous true state uniform in
// the ROI, its NCV successor, a previous posterior mean and a particle around it, the
// observation of the successor (LoS + the given surfaces, random phases common to all PAs
// or drawn per PA, noise of variance eta), the summary at the predicted mean, and the
// target u that carries the
// particle to the true successor (least squares through Gamma).
#include <string>

#include "bp_handle.cuh"

namespace bp {

constexpr double LP_POS_UNIT = 0.01, LP_VEL_UNIT = 0.1, LP_LS_MIN = -4.0, LP_LS_MAX = 1.0;
constexpr int LP_NS = 10;   // shared summary features

// ROI-centred position features and the correlation summary; cor[j] = (Re c, Im c,
// |z_j|^2, |psi_j|^2) with c = psi_j^H z_j
__host__ __device__ inline void lp_shared(const DevParams& Pm, int J, const double* xbar, const double (*cor)[4],
                                          double* f) {
    for (int a = 0; a < 3; ++a) {
        const double c = 0.5 * (Pm.p_min[a] + Pm.p_max[a]);
        const double hw = fmax(0.5 * (Pm.p_max[a] - Pm.p_min[a]), 0.5);
        f[a] = (xbar[a] - c) / hw;
    }
    double rr[4] = {0, 0, 0, 0}, ri[4] = {0, 0, 0, 0};
    for (int j = 0; j < J && j < 4; ++j) {
        const double nn = cor[j][2] * cor[j][3];
        if (nn > 0.0) {
            const double s = 1.0 / sqrt(nn);
            rr[j] = cor[j][0] * s;
            ri[j] = cor[j][1] * s;
        }
    }
    const double r0 = sqrt(rr[0] * rr[0] + ri[0] * ri[0]);
    const double inv0 = 1.0 / fmax(r0, 1e-12);
    for (int j = 1; j < 4; ++j) {
        // rho_j conj(rho_0) / |rho_0|
        f[3 + 2 * (j - 1)] = (rr[j] * rr[0] + ri[j] * ri[0]) * inv0;
        f[4 + 2 * (j - 1)] = (ri[j] * rr[0] - rr[j] * ri[0]) * inv0;
    }
    f[9] = r0;
}

__device__ inline double blk_sum(double v, double* red) {
    const int t = threadIdx.x;
    red[t] = v;
    __syncthreads();
    for (int o = blockDim.x >> 1; o > 0; o >>= 1) {
        if (t < o) red[t] += red[t + o];
        __syncthreads();
    }
    const double r = red[0];
    __syncthreads();
    return r;
}

// lp[0..5] = sum_p w_beta x_n^p / sum_p w_beta (one block of 1024, fixed order)
__global__ void __launch_bounds__(1024) k_lp_mean(DevParams Pm, DevState D, double* lp) {
    __shared__ double red[1024];
    const int P = Pm.P;
    const float* x = D.x[D.cur];
    double s[7] = {0, 0, 0, 0, 0, 0, 0};
    for (int p = threadIdx.x; p < P; p += blockDim.x) {
        const double w = D.w_x[p];
        for (int k = 0; k < 6; ++k) s[k] += w * (double)x[k * P + p];
        s[6] += w;
    }
    double tot[7];
    for (int k = 0; k < 7; ++k) tot[k] = blk_sum(s[k], red);
    if (threadIdx.x < 6) lp[threadIdx.x] = tot[threadIdx.x] / tot[6];
}

// lp[6 + 4 j ..] = (Re, Im of psi_j(xbar)^H z_j, |z_j|^2, |psi_j|^2), FP64, block per PA
__global__ void __launch_bounds__(256) k_lp_corr(DevGeom G, const float* __restrict__ z, double* lp) {
    __shared__ double red[256];
    const int j = blockIdx.x, Nz = G.Nz, Nm = G.My * G.Mz;
    const PathGeo g = path_geo(G, j, lp[0], lp[1], lp[2], 0, 0, 0, true);
    double cr = 0, ci = 0, nz = 0, np = 0;
    for (int k = threadIdx.x; k < Nz; k += blockDim.x) {
        const int f = k / Nm, r = k - f * Nm, y = r / G.Mz, m = r - y * G.Mz;
        const double2 ps = steer_elem(G, g, f, y, m);
        const double zr = z[2 * (j * Nz + k)], zi = z[2 * (j * Nz + k) + 1];
        cr += ps.x * zr + ps.y * zi;
        ci += ps.x * zi - ps.y * zr;
        nz += zr * zr + zi * zi;
        np += ps.x * ps.x + ps.y * ps.y;
    }
    cr = blk_sum(cr, red); ci = blk_sum(ci, red); nz = blk_sum(nz, red); np = blk_sum(np, red);
    if (threadIdx.x == 0) {
        double* o = lp + 6 + 4 * j;
        o[0] = cr; o[1] = ci; o[2] = nz; o[3] = np;
    }
}

// F x_{n-1} of particle p from the predicted particle and the prediction's draws
__device__ inline void lp_prev_mean(const DevParams& Pm, const float* x, int P, int p, int n, double* fx, double* up) {
    float g[3];
    normals8(Pm, p, n, RNG_MT_PREDICT, 0, 3, g);
    const float sv = (float)Pm.sigma_v, T = (float)Pm.T;
    for (int k = 0; k < 3; ++k) {
        const float w = (Pm.motion_dims == 2 && k == 2) ? 0.f : sv * g[k];
        up[k] = (Pm.motion_dims == 2 && k == 2) ? 0.0 : (double)g[k];
        fx[k] = (double)x[k * P + p] - (double)(0.5f * T * T * w);
        fx[3 + k] = (double)x[(3 + k) * P + p] - (double)(T * w);
    }
}

__global__ void k_lp_inputs(DevGeom G, DevParams Pm, DevState D, const double* __restrict__ lp, float* __restrict__ X) {
    const int p = blockIdx.x * blockDim.x + threadIdx.x;
    const int P = Pm.P;
    if (p >= P) return;
    const int n = D.step[0];
    double f[LP_NS];
    lp_shared(Pm, G.J, lp, reinterpret_cast<const double(*)[4]>(lp + 6), f);
    double fx[6], up[3];
    lp_prev_mean(Pm, D.x[D.cur], P, p, n, fx, up);
    float* row = X + (size_t)p * 16;
    for (int k = 0; k < 3; ++k) {
        row[k] = (float)((fx[k] - lp[k]) / LP_POS_UNIT);
        row[3 + k] = (float)((fx[3 + k] - lp[3 + k]) / LP_VEL_UNIT);
    }
    for (int k = 0; k < LP_NS; ++k) row[6 + k] = (float)f[k];
}

// draw from the proposal, move the particle, weight by transition / proposal
__global__ void k_lp_apply(DevParams Pm, DevState D, const float* __restrict__ Y, double* __restrict__ logr) {
    const int p = blockIdx.x * blockDim.x + threadIdx.x;
    const int P = Pm.P;
    if (p >= P) return;
    const int n = D.step[0];
    float* x = D.x[D.cur];
    double fx[6], up[3];
    lp_prev_mean(Pm, x, P, p, n, fx, up);
    float g[3];
    normals8(Pm, p, n, RNG_LEARNED_PROP, 0, 3, g);
    const double T = Pm.T, sv = Pm.sigma_v;
    double lr = 0.0;
    for (int k = 0; k < 3; ++k) {
        if (Pm.motion_dims == 2 && k == 2) continue;
        const double mu = (double)Y[(size_t)p * 16 + k];
        const double ls = fmin(fmax((double)Y[(size_t)p * 16 + 3 + k], LP_LS_MIN), LP_LS_MAX);
        const double u = mu + exp(ls) * (double)g[k];
        lr += -0.5 * u * u + 0.5 * (double)g[k] * (double)g[k] + ls;
        x[k * P + p] = (float)(fx[k] + 0.5 * T * T * sv * u);
        x[(3 + k) * P + p] = (float)(fx[3 + k] + T * sv * u);
    }
    logr[p] = lr;
    D.w_x[p] *= exp(lr);
}

__global__ void __launch_bounds__(1024) k_lp_norm(DevParams Pm, DevState D) {
    __shared__ double red[1024];
    const int P = Pm.P;
    double s = 0.0;
    for (int p = threadIdx.x; p < P; p += blockDim.x) s += D.w_x[p];
    const double tot = blk_sum(s, red);
    const double inv = 1.0 / tot;
    for (int p = threadIdx.x; p < P; p += blockDim.x) D.w_x[p] *= inv;
}

// ---------------------------------------------------------------- training data
struct LpData {
    int K, coherent;
    const double* sfv;      // K x 3
    const double* rho_abs;  // K + 1
    double eta, err_pos, err_vel, spr_pos, spr_vel;
};

constexpr int LP_KMAX = 64;

// per-warp shared memory of the dataset kernel: Kronecker factors b_f, a_y, a_z of the
// K + 1 true components and of the LoS at the predicted mean, for one PA
__host__ __device__ inline int lp_factor_count(const DevGeom& G) { return G.Nf + G.My + G.Mz; }

// one warp per sample
__global__ void k_lp_dataset(DevGeom G, DevParams Pm, LpData L, int nsamp, float* __restrict__ X, float* __restrict__ Tt) {
    extern __shared__ double2 lp_sm[];
    const int lane = threadIdx.x & 31, wib = threadIdx.x >> 5;
    const int i = blockIdx.x * (blockDim.x >> 5) + wib;
    if (i >= nsamp) return;
    const int J = G.J, Nz = G.Nz, Nm = G.My * G.Mz, NFc = lp_factor_count(G), NC = L.K + 2;
    double2* fac = lp_sm + (size_t)wib * NC * NFc;     // [NC][Nf + My + Mz]
    const double T = Pm.T, sv = Pm.sigma_v;
    const bool planar = Pm.motion_dims == 2;
    // scalar draws (every lane computes the same values from the same counters)
    double xp[6], u[3], xh[6], xq[6];
    {
        const U4 a = draw(Pm, i, 0, RNG_LP_DATA, 0, 0), b = draw(Pm, i, 0, RNG_LP_DATA, 0, 1);
        const uint32_t uu[6] = {a.x, a.y, a.z, a.w, b.x, b.y};
        for (int k = 0; k < 3; ++k) {
            xp[k] = Pm.p_min[k] + (Pm.p_max[k] - Pm.p_min[k]) * u24d(uu[k]);
            xp[3 + k] = Pm.v_max[k] * (2.0 * u24d(uu[3 + k]) - 1.0);
        }
        float g[8];
        normals8(Pm, i, 0, RNG_LP_DATA, 1, 3, g);
        for (int k = 0; k < 3; ++k) u[k] = g[k];
        normals8(Pm, i, 0, RNG_LP_DATA, 2, 6, g);
        for (int k = 0; k < 3; ++k) { xh[k] = xp[k] + L.err_pos * g[k]; xh[3 + k] = xp[3 + k] + L.err_vel * g[3 + k]; }
        normals8(Pm, i, 0, RNG_LP_DATA, 3, 6, g);
        for (int k = 0; k < 3; ++k) { xq[k] = xh[k] + L.spr_pos * g[k]; xq[3 + k] = xh[3 + k] + L.spr_vel * g[3 + k]; }
        if (planar) {
            xp[5] = 0.0; u[2] = 0.0;
            xh[2] = xq[2] = xp[2];
            xh[5] = xq[5] = 0.0;
        }
    }
    // true successor, predicted mean, the particle's F x_{n-1}
    double xt[6], xb[6], fq[6];
    for (int k = 0; k < 3; ++k) {
        xt[k] = xp[k] + T * xp[3 + k] + 0.5 * T * T * sv * u[k];
        xt[3 + k] = xp[3 + k] + T * sv * u[k];
        xb[k] = xh[k] + T * xh[3 + k];
        xb[3 + k] = xh[3 + k];
        fq[k] = xq[k] + T * xq[3 + k];
        fq[3 + k] = xq[3 + k];
    }
    // the observation of the successor (LoS + K surfaces + noise) and its summary at xb
    double cor[4][4] = {};
    for (int j = 0; j < J; ++j) {
        // complex amplitudes of the components, applied to the factors b_f: phases common
        // to all PAs (coherent data) or drawn per PA (noncoherent data)
        double amp_r[LP_KMAX + 1], amp_i[LP_KMAX + 1];
        for (int c = 0; c <= L.K; ++c) {
            const U4 pr = draw(Pm, i, 0, RNG_LP_DATA, 4, L.coherent ? c : c + 128 * (j + 1));
            double sp, cp;
            sincospi(2.0 * u24d(pr.x), &sp, &cp);
            amp_r[c] = L.rho_abs[c] * cp;
            amp_i[c] = L.rho_abs[c] * sp;
        }
        // factors of component c (c = K + 1: the LoS at xb): b_f carries the path loss
        // and (for true components) the complex amplitude
        for (int t = lane; t < NC * NFc; t += 32) {
            const int c = t / NFc, q = t - c * NFc;
            const bool los = (c == 0) || (c == L.K + 1);
            const double* sp = (c >= 1 && c <= L.K) ? L.sfv + 3 * (c - 1) : nullptr;
            const double* pp = (c == L.K + 1) ? xb : xt;
            const PathGeo gc = path_geo(G, j, pp[0], pp[1], pp[2], sp ? sp[0] : 0, sp ? sp[1] : 0, sp ? sp[2] : 0, los);
            double2 v;
            if (q < G.Nf) {
                const double2 e = cis_cycles(-(G.fc + G.f[q]) * gc.d / G.c);
                const double a = G.lam / (4.0 * M_PI * gc.d);
                const double ar = (c <= L.K) ? amp_r[c] : 1.0, ai = (c <= L.K) ? amp_i[c] : 0.0;
                v = make_double2(a * (ar * e.x - ai * e.y), a * (ar * e.y + ai * e.x));
            } else if (q < G.Nf + G.My) {
                v = cis_cycles(G.py[q - G.Nf] * gc.uy / G.lam);
            } else {
                v = cis_cycles(G.pz[q - G.Nf - G.My] * gc.uz / G.lam);
            }
            fac[t] = v;
        }
        __syncwarp();
        double cr = 0, ci = 0, nz = 0, np = 0;
        for (int k = lane; k < Nz; k += 32) {
            const int f = k / Nm, r = k - f * Nm, y = r / G.Mz, m = r - y * G.Mz;
            double zr = 0, zi = 0, pr = 0, pi = 0;
            for (int c = 0; c < NC; ++c) {
                const double2* fc = fac + c * NFc;
                const double2 b = fc[f], ay = fc[G.Nf + y], az = fc[G.Nf + G.My + m];
                const double yr = ay.x * az.x - ay.y * az.y, yi = ay.x * az.y + ay.y * az.x;
                const double er = b.x * yr - b.y * yi, ei = b.x * yi + b.y * yr;
                if (c <= L.K) { zr += er; zi += ei; } else { pr = er; pi = ei; }
            }
            float nrm[2];
            normals8(Pm, i, 1 + j * Nz + k, RNG_LP_DATA, 5, 2, nrm);
            const double sn = sqrt(0.5 * L.eta);
            zr += sn * nrm[0];
            zi += sn * nrm[1];
            cr += pr * zr + pi * zi;
            ci += pr * zi - pi * zr;
            nz += zr * zr + zi * zi;
            np += pr * pr + pi * pi;
        }
        cor[j][0] = warp_sum_d(cr);
        cor[j][1] = warp_sum_d(ci);
        cor[j][2] = warp_sum_d(nz);
        cor[j][3] = warp_sum_d(np);
        __syncwarp();
    }
    if (lane != 0) return;
    double f[LP_NS];
    lp_shared(Pm, J, xb, cor, f);
    float* row = X + (size_t)i * 16;
    for (int k = 0; k < 3; ++k) {
        row[k] = (float)((fq[k] - xb[k]) / LP_POS_UNIT);
        row[3 + k] = (float)((fq[3 + k] - xb[3 + k]) / LP_VEL_UNIT);
    }
    for (int k = 0; k < LP_NS; ++k) row[6 + k] = (float)f[k];
    // target: the u that carries the particle to the true successor, least squares
    // through Gamma = [T^2/2 I; T I]
    const double den = (0.25 * T * T * T * T + T * T) * sv;
    for (int k = 0; k < 3; ++k) {
        const double t = (0.5 * T * T * (xt[k] - fq[k]) + T * (xt[3 + k] - fq[3 + k])) / den;
        Tt[(size_t)i * 3 + k] = (float)((planar && k == 2) ? 0.0 : t);
    }
}

}  // namespace bp

using namespace bp;

int launch_learned_proposal(const bp_handle* h, const float* z_dev) {
    if (!h->lp_net) return 0;
    const int P = h->P;
    cudaStream_t st = h->st;
    k_lp_mean<<<1, 1024, 0, st>>>(h->Pm, h->D, h->lp_buf);
    k_lp_corr<<<h->J, 256, 0, st>>>(h->G, z_dev, h->lp_buf);
    k_lp_inputs<<<(P + 255) / 256, 256, 0, st>>>(h->G, h->Pm, h->D, h->lp_buf, h->lp_X);
    mlp_forward_async(h->lp_net, h->lp_X, P, h->lp_Y, st);
    k_lp_apply<<<(P + 255) / 256, 256, 0, st>>>(h->Pm, h->D, h->lp_Y, h->lp_logr);
    k_lp_norm<<<1, 1024, 0, st>>>(h->Pm, h->D);
    return 6;
}


extern "C" {

bp_status bp_set_mt_proposal(bp_handle* h, bp_mlp* net) {
    if (!h) return BP_ERR_INVALID_ARG;
    // handles of a batch (their workspace is the batch's) replay captured graphs that a
    // network attached later would not be part of
    if (!h->ws_owned && net) {
        h->err = "bp_set_mt_proposal: not available on a handle of a batch";
        return BP_ERR_STATE;
    }
    if (net && h->J > 4) {
        h->err = "bp_set_mt_proposal: the proposal summary covers at most 4 PAs";
        return BP_ERR_INVALID_ARG;
    }
    if (net && !h->lp_X) {
        const size_t P = (size_t)h->P;
        if (cudaMalloc(&h->lp_X, P * 16 * sizeof(float)) != cudaSuccess ||
            cudaMalloc(&h->lp_Y, P * 16 * sizeof(float)) != cudaSuccess ||
            cudaMalloc(&h->lp_logr, P * sizeof(double)) != cudaSuccess ||
            cudaMalloc(&h->lp_buf, 32 * sizeof(double)) != cudaSuccess) {
            h->err = "bp_set_mt_proposal: allocation failed";
            return BP_ERR_CUDA;
        }
        h->allocs.push_back(h->lp_X);
        h->allocs.push_back(h->lp_Y);
        h->allocs.push_back(h->lp_logr);
        h->allocs.push_back(h->lp_buf);
    }
    h->lp_net = net;
    return BP_OK;
}

bp_status bp_lp_dataset(const bp_geometry* geom, const bp_params* prm, int K, const double* sfv, const double* rho_abs,
                        double eta, int coherent, double err_pos, double err_vel, double spread_pos, double spread_vel, int n,
                        uint64_t seed, float* X_dev, float* T_dev, void* cuda_stream) {
    if (validate_geom(geom) != BP_OK || !prm || K < 0 || K > LP_KMAX || (K > 0 && !sfv) || !rho_abs || !(eta > 0.0) || n < 1 ||
        !X_dev || !T_dev || !(err_pos >= 0) || !(err_vel >= 0) || !(spread_pos >= 0) || !(spread_vel >= 0) ||
        (prm->motion_dims != 2 && prm->motion_dims != 3) || !(prm->T > 0) || geom->J > 4)
        return BP_ERR_INVALID_ARG;
    DevGeom G;
    fill_geom(G, geom);
    DevParams Pm;
    memset(&Pm, 0, sizeof(Pm));
    Pm.T = prm->T; Pm.sigma_v = prm->sigma_v; Pm.motion_dims = prm->motion_dims;
    for (int k = 0; k < 3; ++k) { Pm.p_min[k] = prm->p_min[k]; Pm.p_max[k] = prm->p_max[k]; Pm.v_max[k] = prm->v_max[k]; }
    Pm.key0 = (uint32_t)(seed & 0xFFFFFFFFu); Pm.key1 = (uint32_t)(seed >> 32);
    cudaStream_t st = static_cast<cudaStream_t>(cuda_stream);
    const size_t smem = (size_t)4 * (K + 2) * lp_factor_count(G) * sizeof(double2);
    if (smem > (size_t)smem_optin()) return BP_ERR_CAPACITY;
    double* buf = nullptr;
    if (cudaMalloc(&buf, (size_t)(3 * K + K + 1) * sizeof(double)) != cudaSuccess) return BP_ERR_CUDA;
    bool ok = (K == 0 || cudaMemcpyAsync(buf, sfv, (size_t)K * 3 * sizeof(double), cudaMemcpyHostToDevice, st) == cudaSuccess) &&
              cudaMemcpyAsync(buf + 3 * K, rho_abs, (size_t)(K + 1) * sizeof(double), cudaMemcpyHostToDevice, st) == cudaSuccess;
    if (ok) {
        LpData L{K, coherent ? 1 : 0, buf, buf + 3 * K, eta, err_pos, err_vel, spread_pos, spread_vel};
        smem_allow_max((const void*)k_lp_dataset);
        k_lp_dataset<<<(n + 3) / 4, 128, smem, st>>>(G, Pm, L, n, X_dev, T_dev);
        ok = cudaGetLastError() == cudaSuccess && cudaStreamSynchronize(st) == cudaSuccess;
    }
    cudaFree(buf);
    return ok ? BP_OK : BP_ERR_CUDA;
}

}  // extern "C"
