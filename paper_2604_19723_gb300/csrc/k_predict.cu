// Initial beliefs, prediction and birth (phase (i) of the message schedule).
//   Sec. V-A: time-0 priors; NCV transition, Gamma(c_eta, eta/c_eta),
//   Gamma(c_gamma, gamma/c_gamma), CN(mu, sigma_mu^2), N(p_sfv, sigma_sfv^2 I).
//   Sec. IV-D: w_beta = w_x, w_xi = w_eta, w_alpha = p_S w_y; births with
//   w_alpha = p_B/P; eq. zeta: zeta(1) = p_S^PR p + p_R^PR (1 - p), new PRs p_B^PR.
#include "bp_internal.cuh"
#include "bp_kernels.cuh"

namespace bp {

// Time-0 beliefs; slots 1 .. S0-1 (if any) are PFs drawn from the birth density over
// the whole birth box, with existence p_B and PR existence p_B^PR like a new PF.
__global__ void k_init(DevGeom G, DevParams Pm, DevState D, int S0) {
    const int p = blockIdx.x * blockDim.x + threadIdx.x;
    const int P = Pm.P;
    if (p < S0 * G.J) D.p_pr[p] = Pm.pB_pr;
    if (p >= P) return;
    float* x = D.x[D.cur];
    float* phi = D.phi[D.cur];
    float* eta = D.eta[D.cur];
    // MT: uniforms 0..5 from blocks 0, 1
    const U4 a = draw(Pm, p, 0, RNG_INIT_MT, 0, 0);
    const U4 b = draw(Pm, p, 0, RNG_INIT_MT, 0, 1);
    const double u[6] = {u24d(a.x), u24d(a.y), u24d(a.z), u24d(a.w), u24d(b.x), u24d(b.y)};
    for (int k = 0; k < 3; ++k) {
        x[k * P + p] = (float)(Pm.p_min[k] + (Pm.p_max[k] - Pm.p_min[k]) * u[k]);
        x[(3 + k) * P + p] = (float)(-Pm.v_max[k] + 2.0 * Pm.v_max[k] * u[3 + k]);
    }
    if (Pm.motion_dims == 2) x[5 * P + p] = 0.0f;
    for (int j = 0; j < G.J; ++j) {
        const U4 e = draw(Pm, p, 0, RNG_INIT_ETA, j, 0);
        eta[j * P + p] = (float)(Pm.eta_min + (Pm.eta_max - Pm.eta_min) * u24d(e.x));
        D.w_eta[j * P + p] = 1.0 / P;
    }
    // LoS drawn like a new PF (birth draws of slot 0 at n = 0)
    const U4 c = draw(Pm, p, 0, RNG_BIRTH, 0, 0);
    const U4 d = draw(Pm, p, 0, RNG_BIRTH, 0, 1);
    phi[0 * P + p] = 0.f; phi[1 * P + p] = 0.f; phi[2 * P + p] = 0.f;
    phi[3 * P + p] = (float)(Pm.gamma_max * u24d(c.w));
    if (Pm.zero_mean) {
        phi[4 * P + p] = 0.f; phi[5 * P + p] = 0.f;
    } else {
        const double r = Pm.mu_max * sqrt(u24d(d.x));
        const double t = 2.0 * u24d(d.y);
        phi[4 * P + p] = (float)(r * cospi(t));
        phi[5 * P + p] = (float)(r * sinpi(t));
    }
    for (int s = 1; s < S0; ++s) {
        const U4 e = draw(Pm, p, 0, RNG_BIRTH, s, 0);
        const U4 f = draw(Pm, p, 0, RNG_BIRTH, s, 1);
        const double v[6] = {u24d(e.x), u24d(e.y), u24d(e.z), u24d(e.w), u24d(f.x), u24d(f.y)};
        float* ph = phi + (size_t)s * 6 * P;
        for (int k = 0; k < 3; ++k) ph[k * P + p] = (float)(2.0 * Pm.p_min[k] + 2.0 * (Pm.p_max[k] - Pm.p_min[k]) * v[k]);
        ph[3 * P + p] = (float)(Pm.gamma_max * v[3]);
        if (Pm.zero_mean) {
            ph[4 * P + p] = 0.f; ph[5 * P + p] = 0.f;
        } else {
            const double r = Pm.mu_max * sqrt(v[4]);
            ph[4 * P + p] = (float)(r * cospi(2.0 * v[5]));
            ph[5 * P + p] = (float)(r * sinpi(2.0 * v[5]));
        }
        D.w_y[(size_t)s * P + p] = Pm.pB / P;
    }
    D.w_x[p] = 1.0 / P;
    D.w_y[p] = Pm.pB / P;
}

// n <- n + 1 at the start of a prediction; the step index lives on the device so that
// a captured step (CUDA graph) draws fresh Philox counters at every replay
__global__ void k_step_advance(DevState D) {
    if (threadIdx.x == 0 && blockIdx.x == 0) D.step[0] += 1;
}

__global__ void k_predict(DevGeom G, DevParams Pm, DevState D, int S_old, int S_new) {
    const int p = blockIdx.x * blockDim.x + threadIdx.x;
    const int n = D.step[0];
    const int P = Pm.P;
    const int J = G.J;
    if (p < S_new * J) {   // zeta of every (s, j)
        const int s = p / J;
        const double pr = D.p_pr[p];
        D.zeta[p] = (s < S_old) ? Pm.pS_pr * pr + Pm.pR_pr * (1.0 - pr) : Pm.pB_pr;
    }
    if (p >= P) return;
    float* x = D.x[D.cur];
    float* phi = D.phi[D.cur];
    float* eta = D.eta[D.cur];
    const float T = (float)Pm.T;
    // MT: x = Phi_a x + Gamma w, w ~ N(0, sigma_v^2 I)
    {
        float g[3];
        normals8(Pm, p, n, RNG_MT_PREDICT, 0, 3, g);
        const float sv = (float)Pm.sigma_v;
        float w[3] = {sv * g[0], sv * g[1], sv * g[2]};
        if (Pm.motion_dims == 2) w[2] = 0.f;
        for (int k = 0; k < 3; ++k) {
            const float pk = x[k * P + p], vk = x[(3 + k) * P + p];
            x[k * P + p] = pk + T * vk + 0.5f * T * T * w[k];
            x[(3 + k) * P + p] = vk + T * w[k];
        }
    }
    // noise variances
    for (int j = 0; j < J; ++j) {
        const double e = (double)eta[j * P + p];
        eta[j * P + p] = (float)gamma_draw(Pm, p, n, RNG_ETA_PREDICT, j, Pm.c_eta, e / Pm.c_eta);
    }
    // legacy PFs
    for (int s = 0; s < S_old; ++s) {
        float g[5];
        normals8(Pm, p, n, RNG_PF_GAUSS, s, 5, g);
        float* ph = phi + (size_t)s * 6 * P;
        if (s > 0) {
            const float ss = (float)Pm.sigma_sfv;
            ph[0 * P + p] += ss * g[0];
            ph[1 * P + p] += ss * g[1];
            if (Pm.motion_dims != 2) ph[2 * P + p] += ss * g[2];
        }
        const double gm = (double)ph[3 * P + p];
        ph[3 * P + p] = (float)gamma_draw(Pm, p, n, RNG_PF_GAMMA, s, Pm.c_gamma, gm / Pm.c_gamma);
        if (Pm.zero_mean) {
            ph[4 * P + p] = 0.f; ph[5 * P + p] = 0.f;
        } else {
            const float sd = (float)(Pm.sigma_mu / sqrt(2.0));
            ph[4 * P + p] += sd * g[3];
            ph[5 * P + p] += sd * g[4];
        }
        D.w_alpha[(size_t)s * P + p] = Pm.pS * D.w_y[(size_t)s * P + p];
    }
    // births: partition q of the birth box (slabs along x)
    for (int s = S_old; s < S_new; ++s) {
        const int q = s - S_old;
        const U4 a = draw(Pm, p, n, RNG_BIRTH, s, 0);
        const U4 b = draw(Pm, p, n, RNG_BIRTH, s, 1);
        const double u[6] = {u24d(a.x), u24d(a.y), u24d(a.z), u24d(a.w), u24d(b.x), u24d(b.y)};
        double lo[3], hi[3];
        for (int k = 0; k < 3; ++k) { lo[k] = 2.0 * Pm.p_min[k]; hi[k] = 2.0 * Pm.p_max[k]; }
        const double width = (hi[0] - lo[0]) / Pm.Q;
        lo[0] = 2.0 * Pm.p_min[0] + q * width;
        hi[0] = lo[0] + width;
        float* ph = phi + (size_t)s * 6 * P;
        for (int k = 0; k < 3; ++k) ph[k * P + p] = (float)(lo[k] + (hi[k] - lo[k]) * u[k]);
        ph[3 * P + p] = (float)(Pm.gamma_max * u[3]);
        if (Pm.zero_mean) {
            ph[4 * P + p] = 0.f; ph[5 * P + p] = 0.f;
        } else {
            const double r = Pm.mu_max * sqrt(u[4]);
            ph[4 * P + p] = (float)(r * cospi(2.0 * u[5]));
            ph[5 * P + p] = (float)(r * sinpi(2.0 * u[5]));
        }
        D.w_alpha[(size_t)s * P + p] = Pm.pB / P;
    }
}

// Per-row FP64 sums: rows 0..S-1 give W_s = sum_p w_alpha, rows S..S+J-1 give
// eta_bar_j = sum_p w_xi eta (the noise-variance prior mean of Sec. S-V).
// One block per row, fixed summation order (deterministic).
__global__ void k_row_sums(DevParams Pm, DevState D, int S, int J) {
    const int row = blockIdx.x;
    const int P = Pm.P;
    double acc = 0.0;
    if (row < S) {
        const double* w = D.w_alpha + (size_t)row * P;
        for (int p = threadIdx.x; p < P; p += blockDim.x) acc += w[p];
    } else {
        const int j = row - S;
        const double* w = D.w_eta + (size_t)j * P;
        const float* e = D.eta[D.cur] + (size_t)j * P;
        for (int p = threadIdx.x; p < P; p += blockDim.x) acc += w[p] * (double)e[p];
    }
    __shared__ double red[32];
    acc = warp_sum_d(acc);
    if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = acc;
    __syncthreads();
    if (threadIdx.x < 32) {
        double v = (threadIdx.x < (blockDim.x >> 5)) ? red[threadIdx.x] : 0.0;
        v = warp_sum_d(v);
        if (threadIdx.x == 0) {
            if (row < S) D.W[row] = v; else D.eta_bar[row - S] = v;
        }
    }
}

void launch_init(const DevGeom& G, const DevParams& Pm, const DevState& D, int S0, cudaStream_t st) {
    const int nthr = max(Pm.P, S0 * G.J);
    k_init<<<(nthr + 255) / 256, 256, 0, st>>>(G, Pm, D, S0);
}

int launch_predict(const DevGeom& G, const DevParams& Pm, const DevState& D, int S_old, int S_new, cudaStream_t st) {
    const int nthr = max(Pm.P, S_new * G.J);
    k_step_advance<<<1, 32, 0, st>>>(D);
    k_predict<<<(nthr + 255) / 256, 256, 0, st>>>(G, Pm, D, S_old, S_new);
    return 2;
}

void launch_row_sums(const DevParams& Pm, const DevState& D, int S, int J, cudaStream_t st) {
    k_row_sums<<<S + J, 512, 0, st>>>(Pm, D, S, J);
}

}  // namespace bp
