// Beliefs, normalisation, estimates, pruning, resampling, regularisation.
//   Sec. IV-D "Beliefs" / Sec. S-III: log w~ = log w_pred + sum_j log(message).
//   Sec. S-IV: C_y,s = sum_p w~_y,s + (1 - W_s) prod_j kappa~(., 0); the PF
//   log-likelihoods here are already relative to prod_j kappa~(., 0), so the
//   null term is log(1 - W_s).  FP64 log-sum-exp throughout.
//   Sec. II-C: MMSE estimates, declaration, pruning (never the LoS).
//   Systematic resampling (Arulampalam et al. 2002, Alg. 2) and Gaussian
//   kernel regularisation with h_opt = (4/(P(d+2)))^(1/(d+4)) (Musso et al. 2001).
#include "bp_internal.cuh"
#include "bp_kernels.cuh"

namespace bp {

// log weight of particle p in belief b, and a pointer to its state dims
struct BeliefView {
    int kind;       // 0 MT, 1 PF, 2 eta
    int index;      // s or j
    int dims;       // 6 or 1
};

__device__ inline BeliefView belief_of(int b, const DevParams& Pm, int J) {
    if (b == 0) return BeliefView{0, 0, 6};
    if (b <= Pm.S_max) return BeliefView{1, b - 1, 6};
    return BeliefView{2, b - 1 - Pm.S_max, 1};
}

__device__ inline double belief_logw(const DevState& D, const BeliefView& v, int P, int p) {
    if (v.kind == 0) return log(D.w_x[p]) + D.lw_x[p];
    if (v.kind == 1) return log(D.w_alpha[(size_t)v.index * P + p]) + D.lw_y[(size_t)v.index * P + p];
    return log(D.w_eta[(size_t)v.index * P + p]) + D.lw_eta[(size_t)v.index * P + p];
}

__device__ inline void belief_state(const DevState& D, const BeliefView& v, int P, int p, double* out) {
    if (v.kind == 0) {
        const float* x = D.x[D.cur];
        for (int k = 0; k < 6; ++k) out[k] = x[(size_t)k * P + p];
    } else if (v.kind == 1) {
        const float* ph = D.phi[D.cur] + (size_t)v.index * 6 * P;
        for (int k = 0; k < 6; ++k) out[k] = ph[(size_t)k * P + p];
    } else {
        out[0] = D.eta[D.cur][(size_t)v.index * P + p];
    }
}

// active beliefs: b in {0} U {1..S} U {1+S_max .. S_max+J}
__device__ inline int active_belief(int a, int S, int S_max) { return a <= S ? a : 1 + S_max + (a - S - 1); }

__global__ void k_norm_max(DevGeom G, DevParams Pm, DevState D, int S, int NB) {
    const int b = active_belief(blockIdx.y, S, Pm.S_max);
    const BeliefView v = belief_of(b, Pm, G.J);
    const int P = Pm.P;
    const int per = (P + NB - 1) / NB;
    const int p0 = blockIdx.x * per, p1 = min(P, p0 + per);
    double m = -INFINITY;
    for (int p = p0 + threadIdx.x; p < p1; p += blockDim.x) m = fmax(m, belief_logw(D, v, P, p));
    __shared__ double red[32];
    m = warp_max_d(m);
    if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = m;
    __syncthreads();
    if (threadIdx.x < 32) {
        double t = threadIdx.x < (blockDim.x >> 5) ? red[threadIdx.x] : -INFINITY;
        t = warp_max_d(t);
        if (threadIdx.x == 0) D.red_part[((size_t)b * NB + blockIdx.x) * RED_W] = t;
    }
}

__global__ void k_norm_sum(DevGeom G, DevParams Pm, DevState D, int S, int NB, double* part) {
    const int b = active_belief(blockIdx.y, S, Pm.S_max);
    const BeliefView v = belief_of(b, Pm, G.J);
    const int P = Pm.P;
    double M = -INFINITY;
    for (int i = 0; i < NB; ++i) M = fmax(M, D.red_part[((size_t)b * NB + i) * RED_W]);
    double ref[6];
    belief_state(D, v, P, 0, ref);
    const int per = (P + NB - 1) / NB;
    const int p0 = blockIdx.x * per, p1 = min(P, p0 + per);
    double acc[RED_W];
    for (int i = 0; i < RED_W; ++i) acc[i] = 0.0;
    const int d = v.dims;
    if (M > -INFINITY) {
        for (int p = p0 + threadIdx.x; p < p1; p += blockDim.x) {
            const double w = exp(belief_logw(D, v, P, p) - M);
            double xs[6];
            belief_state(D, v, P, p, xs);
            for (int k = 0; k < d; ++k) xs[k] -= ref[k];
            acc[0] += w;
            for (int k = 0; k < d; ++k) acc[1 + k] += w * xs[k];
            int t = 7;
            for (int r = 0; r < d; ++r)
                for (int c = r; c < d; ++c) acc[t++] += w * xs[r] * xs[c];
            acc[28] += w * w;
        }
    }
    __shared__ double red[32][RED_W + 1];
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    for (int i = 0; i < RED_W; ++i) {
        const double s = warp_sum_d(acc[i]);
        if (lane == 0) red[wid][i] = s;
    }
    __syncthreads();
    if (threadIdx.x < RED_W) {
        double s = 0.0;
        for (int w = 0; w < (int)(blockDim.x >> 5); ++w) s += red[w][threadIdx.x];
        part[((size_t)b * NB + blockIdx.x) * RED_W + threadIdx.x] = s;
    }
}

__device__ inline void mt_mask(const DevParams& Pm, bool* a) {
    for (int k = 0; k < 6; ++k) a[k] = true;
    if (Pm.motion_dims == 2) { a[2] = false; a[5] = false; }
}
__device__ inline void pf_mask(const DevParams& Pm, int s, bool* a) {
    for (int k = 0; k < 6; ++k) a[k] = true;
    if (s == 0) { a[0] = a[1] = a[2] = false; }
    else if (Pm.motion_dims == 2) a[2] = false;
    if (Pm.zero_mean) { a[4] = a[5] = false; }
}

// one thread per active belief: combine partials, estimates, jitter factor
__global__ void k_norm_final(DevGeom G, DevParams Pm, DevState D, int S, int NB, const double* part) {
    const int a = blockIdx.x * blockDim.x + threadIdx.x;
    if (a >= 1 + S + G.J) return;
    const int b = active_belief(a, S, Pm.S_max);
    const BeliefView v = belief_of(b, Pm, G.J);
    const int P = Pm.P;
    double M = -INFINITY;
    for (int i = 0; i < NB; ++i) M = fmax(M, D.red_part[((size_t)b * NB + i) * RED_W]);
    double acc[RED_W];
    for (int i = 0; i < RED_W; ++i) acc[i] = 0.0;
    for (int i = 0; i < NB; ++i)
        for (int k = 0; k < RED_W; ++k) acc[k] += part[((size_t)b * NB + i) * RED_W + k];
    double ref[6];
    belief_state(D, v, P, 0, ref);
    double* rec = D.bel + bel_rec(Pm.S_max, G.J, b);
    const double lse = (acc[0] > 0) ? M + log(acc[0]) : -INFINITY;
    double logC = lse;
    if (v.kind == 1) {
        const double W = D.W[v.index];
        const double ln = (W < 1.0) ? log1p(-W) : -INFINITY;
        const double mx = fmax(lse, ln);
        logC = (mx == -INFINITY) ? -INFINITY : mx + log(exp(lse - mx) + exp(ln - mx));
        const double ps = (logC == -INFINITY) ? 0.0 : exp(lse - logC);
        D.p_s[v.index] = ps;
    }
    rec[0] = M; rec[1] = lse; rec[2] = logC;
    rec[3] = (acc[0] > 0) ? acc[28] / (acc[0] * acc[0]) : 1.0;   // sum of squared normalised weights
    const int d = v.dims;
    double mean[6] = {0, 0, 0, 0, 0, 0};
    double C[6][6];
    for (int r = 0; r < 6; ++r) for (int c = 0; c < 6; ++c) C[r][c] = 0.0;
    if (acc[0] > 0) {
        for (int k = 0; k < d; ++k) mean[k] = acc[1 + k] / acc[0];
        int t = 7;
        for (int r = 0; r < d; ++r)
            for (int c = r; c < d; ++c) {
                const double cv = acc[t++] / acc[0] - mean[r] * mean[c];
                C[r][c] = C[c][r] = cv;
            }
        for (int k = 0; k < d; ++k) mean[k] += ref[k];
    }
    for (int k = 0; k < 6; ++k) rec[4 + k] = (k < d) ? mean[k] : 0.0;
    // regularisation factor h_opt L (active dimensions only)
    bool act[6];
    if (v.kind == 0) mt_mask(Pm, act);
    else if (v.kind == 1) pf_mask(Pm, v.index, act);
    else { act[0] = true; for (int k = 1; k < 6; ++k) act[k] = false; }
    int dact = 0;
    for (int k = 0; k < d; ++k) if (act[k]) ++dact;
    for (int r = 0; r < 6; ++r) for (int c = 0; c < 6; ++c) if (!(r < d && c < d && act[r] && act[c])) C[r][c] = 0.0;
    double L[6][6];
    for (int r = 0; r < 6; ++r) for (int c = 0; c < 6; ++c) L[r][c] = 0.0;
    for (int k = 0; k < d; ++k) {
        double piv = C[k][k];
        for (int m = 0; m < k; ++m) piv -= L[k][m] * L[k][m];
        if (piv <= 0.0) continue;
        L[k][k] = sqrt(piv);
        for (int i = k + 1; i < d; ++i) {
            double s = C[i][k];
            for (int m = 0; m < k; ++m) s -= L[i][m] * L[k][m];
            L[i][k] = s / L[k][k];
        }
    }
    const double h = (dact > 0) ? pow(4.0 / (P * (dact + 2.0)), 1.0 / (dact + 4.0)) : 0.0;
    float* Lf = D.Lchol + (size_t)b * 36;
    for (int r = 0; r < 6; ++r) for (int c = 0; c < 6; ++c) Lf[r * 6 + c] = (float)((Pm.regularize ? h : 0.0) * L[r][c]);
    rec[10] = dact;
}

// estimates, declaration, pruning map; single thread
__global__ void k_estimate(DevGeom G, DevParams Pm, DevState D, int S) {
    if (threadIdx.x != 0 || blockIdx.x != 0) return;
    const int n = D.step[0];
    const int J = G.J, SM = Pm.S_max;
    const EstLayout E{SM, J};
    double* est = D.est;
    est[E.n()] = n;
    est[E.S()] = S;
    est[E.repaired()] = D.flags[0];
    const double* r0 = D.bel + bel_rec(SM, J, 0);
    for (int k = 0; k < 6; ++k) est[E.x_hat() + k] = r0[4 + k];
    est[E.ess()] = 1.0 / r0[3];
    for (int j = 0; j < J; ++j) est[E.eta_hat() + j] = (D.bel + bel_rec(SM, J, 1 + SM + j))[4];
    int keep = 0;
    for (int s = 0; s < S; ++s) {
        const double* rs = D.bel + bel_rec(SM, J, 1 + s);
        const double ps = D.p_s[s];
        est[E.p_s() + s] = ps;
        for (int k = 0; k < 6; ++k) est[E.phi_hat() + 6 * s + k] = rs[4 + k];
        double prod = 1.0;
        for (int j = 0; j < J; ++j) {
            const double pr = D.bel[BEL_PPR + s * J + j];
            est[E.p_pr() + s * J + j] = pr;
            prod *= (1.0 - pr);
        }
        const double pany = 1.0 - prod;
        est[E.p_any() + s] = pany;
        est[E.declared() + s] = (ps > Pm.T_dec) ? 1.0 : 0.0;
        const bool kept = (s == 0) || Pm.T_pru <= 0.0 || !(ps < Pm.T_pru || pany < Pm.T_pru);
        if (kept) D.ctrl[4 + keep++] = s;
    }
    D.ctrl[1] = keep;
    est[E.S_next()] = keep;
    est[E.skipped()] = D.ctrl[2];
    int status = 0;
    if (!(r0[2] > -INFINITY)) status = BP_ERR_NUMERIC;
    // a NaN or Inf in z reaches |e|^2 of its PA first; report it as such
    for (int j = 0; j < J; ++j)
        if (!isfinite(D.nu_c[2 * j])) status = EST_STATUS_BAD_Z;
    est[E.status()] = status;
    D.ctrl[3] = status;
}

// normalised weights of every active belief (before resampling)
__global__ void k_norm_weights(DevGeom G, DevParams Pm, DevState D, int S) {
    const int P = Pm.P;
    const int b = active_belief(blockIdx.y, S, Pm.S_max);
    const BeliefView v = belief_of(b, Pm, G.J);
    const double logC = (D.bel + bel_rec(Pm.S_max, G.J, b))[2];
    for (int p = blockIdx.x * blockDim.x + threadIdx.x; p < P; p += gridDim.x * blockDim.x) {
        const double w = (logC > -INFINITY) ? exp(belief_logw(D, v, P, p) - logC) : 0.0;
        if (v.kind == 0) D.wn_x[p] = w;
        else if (v.kind == 1) D.wn_y[(size_t)v.index * P + p] = w;
        else D.wn_eta[(size_t)v.index * P + p] = w;
    }
}

int launch_normalize(const DevGeom& G, const DevParams& Pm, const DevState& D, int S, cudaStream_t st) {
    const int P = Pm.P;
    int NB = (P + 4095) / 4096;
    if (NB > 64) NB = 64;
    const int nb = 1 + S + G.J;
    double* part = D.red_part + (size_t)bel_count(Pm.S_max, G.J) * 64 * RED_W;
    k_norm_max<<<dim3(NB, nb), 256, 0, st>>>(G, Pm, D, S, NB);
    k_norm_sum<<<dim3(NB, nb), 256, 0, st>>>(G, Pm, D, S, NB, part);
    k_norm_final<<<(nb + 63) / 64, 64, 0, st>>>(G, Pm, D, S, NB, part);
    k_estimate<<<1, 32, 0, st>>>(G, Pm, D, S);
    k_norm_weights<<<dim3((P + 255) / 256 < 256 ? (P + 255) / 256 : 256, nb), 256, 0, st>>>(G, Pm, D, S);
    return 5;
}

// ---------------------------------------------------------------- systematic resampling
// one block per kept belief; CDF in FP64 (chunked per thread, block exclusive scan)
__global__ void __launch_bounds__(1024) k_resample(DevGeom G, DevParams Pm, DevState D, int S, double* cdf_all) {
    const int P = Pm.P, SM = Pm.S_max, J = G.J;
    const int n = D.step[0];
    const int S_next = D.ctrl[1];
    const int a = blockIdx.x;   // 0: MT, 1..S_next: kept PF, then eta
    int b, kind, index;
    if (a == 0) { b = 0; kind = 0; index = 0; }
    else if (a <= S_next) {
        index = D.ctrl[4 + a - 1]; b = 1 + index; kind = 1;
        if (!bp_in_range(index, SM, D.kerr)) return;
    }
    else if (a <= S_next + J) { index = a - S_next - 1; b = 1 + SM + index; kind = 2; }
    else return;
    const double* w = (kind == 0) ? D.wn_x : (kind == 1) ? D.wn_y + (size_t)index * P : D.wn_eta + (size_t)index * P;
    double* cdf = cdf_all + (size_t)a * P;
    const int per = (P + blockDim.x - 1) / blockDim.x;
    const int p0 = threadIdx.x * per, p1 = min(P, p0 + per);
    double loc = 0.0;
    for (int p = p0; p < p1; ++p) loc += w[p];
    __shared__ double scan[1024];
    __shared__ double total;
    scan[threadIdx.x] = loc;
    __syncthreads();
    for (int off = 1; off < (int)blockDim.x; off <<= 1) {
        const double t = (threadIdx.x >= (unsigned)off) ? scan[threadIdx.x - off] : 0.0;
        __syncthreads();
        scan[threadIdx.x] += t;
        __syncthreads();
    }
    if (threadIdx.x == blockDim.x - 1) total = scan[threadIdx.x];
    __syncthreads();
    double run = scan[threadIdx.x] - loc;
    for (int p = p0; p < p1; ++p) { run += w[p]; cdf[p] = run; }
    __syncthreads();
    const double tot = total;
    for (int p = p0; p < p1; ++p) cdf[p] = (tot > 0) ? cdf[p] / tot : (double)(p + 1) / P;
    __syncthreads();
    if (threadIdx.x == 0) cdf[P - 1] = 1.0;
    __syncthreads();
    const U4 r = draw(Pm, (uint32_t)((kind << 16) | index), n, RNG_RESAMPLE, 0, 0);
    const double U = u32d(r.x);
    int* idx = D.idx + (size_t)b * P;
    for (int i = threadIdx.x; i < P; i += blockDim.x) {
        const double u = (U + (double)i) / (double)P;
        int lo = 0, hi = P - 1;            // first k with cdf[k] >= u
        while (lo < hi) {
            const int mid = (lo + hi) >> 1;
            if (cdf[mid] >= u) hi = mid; else lo = mid + 1;
        }
        idx[i] = lo;
    }
}

// gather + jitter into the other buffer; thread per output slot
__global__ void k_gather(DevGeom G, DevParams Pm, DevState D) {
    const int P = Pm.P, SM = Pm.S_max, J = G.J;
    const int n = D.step[0];
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    const int S_next = D.ctrl[1];
    const int nxt = 1 - D.cur;
    if (i < P) {
        {   // MT
            int src = D.idx[i];
            if (!bp_in_range(src, P, D.kerr)) src = i;
            const float* L = D.Lchol;
            float e[6];
            normals8(Pm, i, n, RNG_JITTER_MT, 0, 6, e);
            for (int r = 0; r < 6; ++r) {
                float jit = 0.f;
                for (int c = 0; c <= r; ++c) jit += L[r * 6 + c] * e[c];
                D.x[nxt][(size_t)r * P + i] = D.x[D.cur][(size_t)r * P + src] + jit;
            }
            D.w_x[i] = 1.0 / P;
        }
        for (int t = 0; t < S_next; ++t) {
            const int s = D.ctrl[4 + t];
            if (!bp_in_range(s, SM, D.kerr)) continue;
            int src = D.idx[(size_t)(1 + s) * P + i];
            if (!bp_in_range(src, P, D.kerr)) src = i;
            const float* L = D.Lchol + (size_t)(1 + s) * 36;
            float e[6];
            normals8(Pm, i, n, RNG_JITTER_PF, s, 6, e);
            const float* ph = D.phi[D.cur] + (size_t)s * 6 * P;
            float* po = D.phi[nxt] + (size_t)t * 6 * P;
            for (int r = 0; r < 6; ++r) {
                float jit = 0.f;
                for (int c = 0; c <= r; ++c) jit += L[r * 6 + c] * e[c];
                float v = ph[(size_t)r * P + src] + jit;
                if (r == 3) v = fabsf(v);
                po[(size_t)r * P + i] = v;
            }
        }
        for (int j = 0; j < J; ++j) {
            int src = D.idx[(size_t)(1 + SM + j) * P + i];
            if (!bp_in_range(src, P, D.kerr)) src = i;
            const float L = D.Lchol[(size_t)(1 + SM + j) * 36];
            float e[1];
            normals8(Pm, i, n, RNG_JITTER_ETA, j, 1, e);
            D.eta[nxt][(size_t)j * P + i] = fabsf(D.eta[D.cur][(size_t)j * P + src] + L * e[0]);
            D.w_eta[(size_t)j * P + i] = 1.0 / P;
        }
    }
}

// weights and PR tables of the compacted PF set; runs after k_gather (reads p_s, writes w_y)
__global__ void k_compact(DevGeom G, DevParams Pm, DevState D) {
    const int P = Pm.P, J = G.J;
    const int S_next = D.ctrl[1];
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    __shared__ double ps_new[S_CAP_MAX];
    if (threadIdx.x < S_next && bp_in_range(D.ctrl[4 + threadIdx.x], Pm.S_max, D.kerr))
        ps_new[threadIdx.x] = D.p_s[D.ctrl[4 + threadIdx.x]];
    __syncthreads();
    if (i < P)
        for (int t = 0; t < S_next; ++t) D.w_y[(size_t)t * P + i] = ps_new[t] / P;
    if (blockIdx.x == 0)
        for (int u = threadIdx.x; u < S_next * J; u += blockDim.x) {
            const int t = u / J, j = u - t * J;
            if (bp_in_range(D.ctrl[4 + t], Pm.S_max, D.kerr)) D.p_pr[t * J + j] = D.bel[BEL_PPR + D.ctrl[4 + t] * J + j];
        }
}

void launch_resample(const DevGeom& G, const DevParams& Pm, const DevState& D, int S, double* cdf, cudaStream_t st) {
    const int nb = 1 + S + G.J;
    k_resample<<<nb, 1024, 0, st>>>(G, Pm, D, S, cdf);
    k_gather<<<(Pm.P + 255) / 256, 256, 0, st>>>(G, Pm, D);
    k_compact<<<(Pm.P + 255) / 256, 256, 0, st>>>(G, Pm, D);
}

}  // namespace bp
