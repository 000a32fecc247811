// Birth proposal PDF (Sec. IV-D, "An Efficient Birth Proposal PDF"), at the start of an
// update (it needs the observation): the residual of z after projecting out the LoS and
// legacy PFs, the coherent Bartlett spectrum at N_g candidates uniform in each new PF's
// partition, the mode-matched mean and moment-matched covariance, and the new PF's
// particles drawn from the Gaussian with importance weights 1_P / proposal density.
//
// Everything that decides the argmax runs in FP64 (one step's worth of work: J
// projections and Q x N_g x J x Nz complex terms); reductions run in a fixed order.
#include "bp_internal.cuh"
#include "bp_kernels.cuh"

namespace bp {

__device__ inline double block_sum_d(double v, double* red) {
    // fixed-order tree over the block (blockDim.x a power of two, <= 1024)
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

// block 0: predicted MT mean (weights w_beta = w_x); block 1 + s: position mean of legacy
// PF s under its prediction weights w_alpha (plain mean if they sum to 0)
__global__ void __launch_bounds__(512) k_bprop_means(DevParams Pm, DevState D, BpropLayout B) {
    __shared__ double red[512];
    const int P = Pm.P, b = blockIdx.x;
    const float* x = D.x[D.cur];
    const float* ph = D.phi[D.cur] + (size_t)(b > 0 ? b - 1 : 0) * 6 * P;
    const double* w = (b == 0) ? D.w_x : D.w_alpha + (size_t)(b - 1) * P;
    const float* src = (b == 0) ? x : ph;
    double a[4] = {0.0, 0.0, 0.0, 0.0};
    for (int p = threadIdx.x; p < P; p += blockDim.x) {
        const double wp = w[p];
        a[0] += wp;
        for (int k = 0; k < 3; ++k) a[1 + k] += wp * (double)src[k * P + p];
    }
    double s[4];
    for (int k = 0; k < 4; ++k) s[k] = block_sum_d(a[k], red);
    if (!(s[0] > 0.0)) {   // no existence mass: plain mean
        double c[3] = {0.0, 0.0, 0.0};
        for (int p = threadIdx.x; p < P; p += blockDim.x)
            for (int k = 0; k < 3; ++k) c[k] += (double)src[k * P + p];
        for (int k = 0; k < 3; ++k) s[1 + k] = block_sum_d(c[k], red);
        s[0] = (double)P;
    }
    if (threadIdx.x == 0)
        for (int k = 0; k < 3; ++k) D.bprop[B.means() + 3 * b + k] = s[1 + k] / s[0];
}

// one block per PA: Psi_j (columns LoS, legacy PFs) at the estimates, Gram and Psi^H z,
// Cholesky (columns whose pivot falls below 1e-12 of their norm are left out: the
// projector onto the column space is the same), z~ = z - Psi c
__global__ void __launch_bounds__(256) k_bprop_resid(DevGeom G, DevState D, BpropLayout B, int S_L, const float* z) {
    extern __shared__ double2 sres[];
    const int j = blockIdx.x, Nz = G.Nz, Nm = G.My * G.Mz;
    double2* gram = sres;                       // [S_L][S_L]
    double2* rhs = gram + (size_t)S_L * S_L;     // [S_L]
    double2* psi = D.bprop_c + B.psi(j);         // [S_L][Nz] (global scratch)
    const double* mean = D.bprop + B.means();
    const double mx = mean[0], my = mean[1], mz = mean[2];
    for (int t = threadIdx.x; t < S_L * Nz; t += blockDim.x) {
        const int s = t / Nz, k = t - s * Nz;
        const int f = k / Nm, ym = k - f * Nm, y = ym / G.Mz, m = ym - y * G.Mz;
        const double* ps = mean + 3 * (1 + s);
        const PathGeo g = path_geo(G, j, mx, my, mz, ps[0], ps[1], ps[2], s == 0);
        psi[t] = steer_elem(G, g, f, y, m);
    }
    __syncthreads();
    const float* zj = z + 2 * (size_t)j * Nz;
    // warp per dot product (lanes over the elements, butterfly sum): G_ac = psi_a^H psi_c
    // for a >= c, then (Psi^H z)_a
    const int lane = threadIdx.x & 31, nw = blockDim.x >> 5;
    const int npair = S_L * (S_L + 1) / 2;
    for (int t = threadIdx.x >> 5; t < npair + S_L; t += nw) {
        double2 acc = make_double2(0.0, 0.0);
        if (t < npair) {
            int a = 0;
            while ((a + 1) * (a + 2) / 2 <= t) ++a;
            const int c = t - a * (a + 1) / 2;
            const double2* pa = psi + (size_t)a * Nz;
            const double2* pc = psi + (size_t)c * Nz;
            for (int k = lane; k < Nz; k += 32) {
                acc.x += pa[k].x * pc[k].x + pa[k].y * pc[k].y;
                acc.y += pa[k].x * pc[k].y - pa[k].y * pc[k].x;
            }
            for (int o = 16; o > 0; o >>= 1) {
                acc.x += __shfl_xor_sync(0xffffffffu, acc.x, o);
                acc.y += __shfl_xor_sync(0xffffffffu, acc.y, o);
            }
            if (lane == 0) gram[a * S_L + c] = acc;
        } else {
            const int a = t - npair;
            const double2* pa = psi + (size_t)a * Nz;
            for (int k = lane; k < Nz; k += 32) {
                const double zr = zj[2 * k], zi = zj[2 * k + 1];
                acc.x += pa[k].x * zr + pa[k].y * zi;
                acc.y += pa[k].x * zi - pa[k].y * zr;
            }
            for (int o = 16; o > 0; o >>= 1) {
                acc.x += __shfl_xor_sync(0xffffffffu, acc.x, o);
                acc.y += __shfl_xor_sync(0xffffffffu, acc.y, o);
            }
            if (lane == 0) rhs[a] = acc;
        }
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        // in-place Cholesky G = L L^H (lower), then L y = rhs, L^H c = y (c in rhs)
        for (int k = 0; k < S_L; ++k) {
            double piv = gram[k * S_L + k].x;
            for (int i = 0; i < k; ++i) {
                const double2 l = gram[k * S_L + i];
                piv -= l.x * l.x + l.y * l.y;
            }
            const double nrm = gram[k * S_L + k].x;   // untouched diagonal above: G_kk
            const bool keep = piv > 1e-12 * nrm && piv > 0.0;
            const double lkk = keep ? sqrt(piv) : 0.0;
            for (int i = k + 1; i < S_L; ++i) {
                double2 v = gram[i * S_L + k];
                for (int m = 0; m < k; ++m) {
                    const double2 a = gram[i * S_L + m], b = gram[k * S_L + m];   // a conj(b)
                    v.x -= a.x * b.x + a.y * b.y;
                    v.y -= a.y * b.x - a.x * b.y;
                }
                gram[i * S_L + k] = keep ? make_double2(v.x / lkk, v.y / lkk) : make_double2(0.0, 0.0);
            }
            // L_kk kept in the diagonal's imaginary slot (the real part still reads G_kk)
            gram[k * S_L + k].y = lkk;
        }
        for (int k = 0; k < S_L; ++k) {
            const double lkk = gram[k * S_L + k].y;
            double2 v = rhs[k];
            for (int m = 0; m < k; ++m) {
                const double2 a = gram[k * S_L + m], b = rhs[m];
                v.x -= a.x * b.x - a.y * b.y;
                v.y -= a.x * b.y + a.y * b.x;
            }
            rhs[k] = lkk > 0.0 ? make_double2(v.x / lkk, v.y / lkk) : make_double2(0.0, 0.0);
        }
        for (int k = S_L - 1; k >= 0; --k) {
            const double lkk = gram[k * S_L + k].y;
            double2 v = rhs[k];
            for (int m = k + 1; m < S_L; ++m) {
                const double2 a = gram[m * S_L + k], b = rhs[m];   // conj(L_mk) c_m
                v.x -= a.x * b.x + a.y * b.y;
                v.y -= a.x * b.y - a.y * b.x;
            }
            rhs[k] = lkk > 0.0 ? make_double2(v.x / lkk, v.y / lkk) : make_double2(0.0, 0.0);
        }
    }
    __syncthreads();
    double2* zr = D.bprop_c + B.zres(j);
    for (int k = threadIdx.x; k < Nz; k += blockDim.x) {
        double2 v = make_double2(zj[2 * k], zj[2 * k + 1]);
        for (int s = 0; s < S_L; ++s) {
            const double2 a = psi[(size_t)s * Nz + k], c = rhs[s];
            v.x -= a.x * c.x - a.y * c.y;
            v.y -= a.x * c.y + a.y * c.x;
        }
        zr[k] = v;
    }
}

// partition q of the birth box U(2 p_min, 2 p_max): slabs along x
__device__ inline void partition(const DevParams& Pm, int q, double lo[3], double hi[3]) {
    for (int k = 0; k < 3; ++k) { lo[k] = 2.0 * Pm.p_min[k]; hi[k] = 2.0 * Pm.p_max[k]; }
    const double width = (hi[0] - lo[0]) / Pm.Q;
    lo[0] = 2.0 * Pm.p_min[0] + q * width;
    hi[0] = lo[0] + width;
}

// warp per (candidate, partition): candidate position, c_i = |sum_j z~_j^H psi_j(x_hat, p_i) / Nz|^2.
// Lanes take the (PA, antenna element) pairs; psi_{f,y,m} = A b_f a_y a_z with the equally
// spaced frequencies as an FP64 recurrence b_f = b_0 r^f (error ~f 1e-16); the coherent sum
// is a warp reduction in a fixed order.
__global__ void __launch_bounds__(256) k_bprop_bartlett(DevGeom G, DevParams Pm, DevState D, BpropLayout B) {
    const int q = blockIdx.y, Ng = Pm.N_g, Nz = G.Nz, Nm = G.My * G.Mz, Nf = G.Nf;
    const int n = D.step[0];
    const int lane = threadIdx.x & 31;
    const int i = blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5);
    if (i >= Ng) return;
    double lo[3], hi[3];
    partition(Pm, q, lo, hi);
    const U4 u = draw(Pm, (uint32_t)i, (uint32_t)n, RNG_BIRTH_CAND, (uint32_t)q, 0);
    const double cx = lo[0] + (hi[0] - lo[0]) * u24d(u.x);
    const double cy = lo[1] + (hi[1] - lo[1]) * u24d(u.y);
    const double cz = lo[2] + (hi[2] - lo[2]) * u24d(u.z);
    const double* mean = D.bprop + B.means();
    const double df = (Nf > 1) ? (G.f[Nf - 1] - G.f[0]) / (Nf - 1) : 0.0;
    // per PA (lanes j): path geometry, b_0 and the frequency step r, shared by the warp
    __shared__ double gw[8][J_MAX][7];
    double (*gj)[7] = gw[threadIdx.x >> 5];
    for (int j = lane; j < G.J; j += 32) {
        const PathGeo g = path_geo(G, j, mean[0], mean[1], mean[2], cx, cy, cz, false);
        const double2 b0 = cis_cycles(-G.f[0] * g.d / G.c), r = cis_cycles(-df * g.d / G.c);
        gj[j][0] = g.d; gj[j][1] = g.uy; gj[j][2] = g.uz;
        gj[j][3] = b0.x; gj[j][4] = b0.y; gj[j][5] = r.x; gj[j][6] = r.y;
    }
    __syncwarp();
    double2 acc = make_double2(0.0, 0.0);
    for (int t = lane; t < G.J * Nm; t += 32) {
        const int j = t / Nm, ym = t - j * Nm, y = ym / G.Mz, m = ym - y * G.Mz;
        const PathGeo g{gj[j][0], 0.0, gj[j][1], gj[j][2]};
        const double2* zr = D.bprop_c + B.zres(j);
        const double2 r = make_double2(gj[j][5], gj[j][6]);
        double2 b = make_double2(gj[j][3], gj[j][4]), sf = make_double2(0.0, 0.0);
        for (int f = 0; f < Nf; ++f) {
            const double2 zc = zr[f * Nm + ym];        // conj(z) b_f
            sf.x += zc.x * b.x + zc.y * b.y;
            sf.y += zc.x * b.y - zc.y * b.x;
            b = make_double2(b.x * r.x - b.y * r.y, b.x * r.y + b.y * r.x);
        }
        // A a_y a_z = lambda/(4 pi d) exp(j 2 pi (-fc d / c + (p_y uy + p_z uz) / lambda))
        const double amp = G.lam / (4.0 * M_PI * g.d) / Nz;
        const double2 a = cis_cycles(-G.fc * g.d / G.c + (G.py[y] * g.uy + G.pz[m] * g.uz) / G.lam);
        acc.x += amp * (a.x * sf.x - a.y * sf.y);
        acc.y += amp * (a.x * sf.y + a.y * sf.x);
    }
    for (int o = 16; o > 0; o >>= 1) {
        acc.x += __shfl_xor_sync(0xffffffffu, acc.x, o);
        acc.y += __shfl_xor_sync(0xffffffffu, acc.y, o);
    }
    if (lane == 0) {
        const size_t o = (size_t)q * Ng + i;
        D.bprop[B.costs() + o] = acc.x * acc.x + acc.y * acc.y;
        double* cd = D.bprop + B.cand() + 3 * o;
        cd[0] = cx; cd[1] = cy; cd[2] = cz;
    }
}

// one block per partition: sum and first argmax of the costs, mu = p_{i*}, the weighted
// second moment C about mu, its zeroing Cholesky factor
__global__ void __launch_bounds__(1024) k_bprop_moments(DevParams Pm, DevState D, BpropLayout B) {
    __shared__ double red[1024];
    __shared__ int ired[1024];
    const int q = blockIdx.x, Ng = Pm.N_g, t = threadIdx.x;
    const double* c = D.bprop + B.costs() + (size_t)q * Ng;
    const double* cd = D.bprop + B.cand() + (size_t)q * Ng * 3;
    double sum = 0.0, best = -1.0;
    int bi = Ng;
    for (int i = t; i < Ng; i += blockDim.x) {
        sum += c[i];
        if (c[i] > best) { best = c[i]; bi = i; }
    }
    const double tot = block_sum_d(sum, red);
    red[t] = best;
    ired[t] = bi;
    __syncthreads();
    for (int o = blockDim.x >> 1; o > 0; o >>= 1) {
        if (t < o) {
            const double v = red[t + o];
            const int vi = ired[t + o];
            if (v > red[t] || (v == red[t] && vi < ired[t])) { red[t] = v; ired[t] = vi; }
        }
        __syncthreads();
    }
    const int istar = ired[0];
    __syncthreads();
    double* st = D.bprop + B.stats(q);
    const bool valid = tot > 0.0 && isfinite(tot) && istar < Ng;
    double mu[3] = {0.0, 0.0, 0.0};
    if (valid)
        for (int k = 0; k < 3; ++k) mu[k] = cd[3 * istar + k];
    double m[6] = {0.0, 0.0, 0.0, 0.0, 0.0, 0.0};   // xx, yx, yy, zx, zy, zz
    if (valid)
        for (int i = t; i < Ng; i += blockDim.x) {
            const double w = c[i] / tot;
            const double d0 = cd[3 * i] - mu[0], d1 = cd[3 * i + 1] - mu[1], d2 = cd[3 * i + 2] - mu[2];
            m[0] += w * d0 * d0; m[1] += w * d1 * d0; m[2] += w * d1 * d1;
            m[3] += w * d2 * d0; m[4] += w * d2 * d1; m[5] += w * d2 * d2;
        }
    double Cm[6];
    for (int k = 0; k < 6; ++k) Cm[k] = block_sum_d(m[k], red);
    if (t == 0) {
        const double C[3][3] = {{Cm[0], Cm[1], Cm[3]}, {Cm[1], Cm[2], Cm[4]}, {Cm[3], Cm[4], Cm[5]}};
        double L[3][3] = {{0.0, 0.0, 0.0}, {0.0, 0.0, 0.0}, {0.0, 0.0, 0.0}};
        for (int k = 0; k < 3; ++k) {
            double piv = C[k][k];
            for (int i = 0; i < k; ++i) piv -= L[k][i] * L[k][i];
            if (piv <= 0.0) continue;   // zero column: no spread along this direction
            L[k][k] = sqrt(piv);
            for (int i = k + 1; i < 3; ++i) {
                double v = C[i][k];
                for (int mm = 0; mm < k; ++mm) v -= L[i][mm] * L[k][mm];
                L[i][k] = v / L[k][k];
            }
        }
        st[0] = valid ? 1.0 : 0.0;
        st[1] = (double)(valid ? istar : -1);
        st[2] = tot;
        for (int k = 0; k < 3; ++k) st[3 + k] = mu[k];
        for (int r = 0; r < 3; ++r)
            for (int k = 0; k < 3; ++k) {
                st[6 + 3 * r + k] = C[r][k];
                st[15 + 3 * r + k] = L[r][k];
            }
    }
}

// thread per particle: positions of every new PF from its proposal, unnormalised weights
// 1_P(p) exp(|g_A|^2 / 2) (A: directions with a positive pivot)
// (256 threads per block; per new PF one partial sum of the weights per block)
__global__ void __launch_bounds__(256) k_bprop_draw(DevParams Pm, DevState D, BpropLayout B, int S_L, int S_new) {
    __shared__ double red[256];
    const int p = blockIdx.x * blockDim.x + threadIdx.x;
    const int P = Pm.P;
    const int n = D.step[0];
    for (int s = S_L; s < S_new; ++s) {
        const int q = s - S_L;
        const double* st = D.bprop + B.stats(q);
        if (st[0] == 0.0) continue;
        double wp = 0.0;
        if (p < P) {
            float g[3];
            normals8(Pm, p, n, RNG_BIRTH_PROP, s, 3, g);
            double lo[3], hi[3];
            partition(Pm, q, lo, hi);
            double pos[3];
            bool inside = true;
            double m2 = 0.0;
            for (int r = 0; r < 3; ++r) {
                double v = st[3 + r];
                for (int k = 0; k <= r; ++k) v += st[15 + 3 * r + k] * (double)g[k];
                pos[r] = v;
                inside = inside && v >= lo[r] && v <= hi[r];
                if (st[15 + 4 * r] > 0.0) m2 += (double)g[r] * (double)g[r];
            }
            wp = inside ? exp(0.5 * m2) : 0.0;
            D.w_alpha[(size_t)s * P + p] = wp;
            // the birth-density draws stay in place until the weights are known to be
            // usable (k_bprop_finish)
            double* keep = D.bprop + B.pos(q) + 3 * (size_t)p;
            keep[0] = pos[0]; keep[1] = pos[1]; keep[2] = pos[2];
        }
        const double bs = block_sum_d(wp, red);
        if (threadIdx.x == 0) D.bprop[B.parts(q) + blockIdx.x] = bs;
    }
}

// thread per (particle, new PF): the weights' total from the draw kernel's partials (fixed
// order); if positive the proposal draws replace the birth-density ones and the weights
// are scaled to sum to p_B, otherwise the PF keeps its birth-density draws with weights p_B / P
__global__ void k_bprop_finish(DevParams Pm, DevState D, BpropLayout B, int S_L, int nparts) {
    const int q = blockIdx.y, s = S_L + q, P = Pm.P;
    const int p = blockIdx.x * blockDim.x + threadIdx.x;
    const double* st = D.bprop + B.stats(q);
    if (st[0] == 0.0 || p >= P) return;
    double tot = 0.0;
    const double* part = D.bprop + B.parts(q);
    for (int b = 0; b < nparts; ++b) tot += part[b];
    double* wa = D.w_alpha + (size_t)s * P;
    if (tot > 0.0 && isfinite(tot)) {
        wa[p] = Pm.pB * (wa[p] / tot);
        float* ph = D.phi[D.cur] + (size_t)s * 6 * P;
        const double* pos = D.bprop + B.pos(q) + 3 * (size_t)p;
        for (int k = 0; k < 3; ++k) ph[k * P + p] = (float)pos[k];
    } else {
        wa[p] = Pm.pB / P;
    }
}

int launch_birth_proposal(const DevGeom& G, const DevParams& Pm, const DevState& D, int S_L, int S_new,
                          const float* z, cudaStream_t st) {
    if (!Pm.birth_proposal || S_new <= S_L || !D.bprop) return 0;
    const BpropLayout B = bprop_layout(G, Pm);
    const int Qe = S_new - S_L;
    k_bprop_means<<<1 + S_L, 512, 0, st>>>(Pm, D, B);
    const size_t sm = ((size_t)S_L * S_L + S_L) * sizeof(double2);
    smem_allow_max((const void*)k_bprop_resid);
    k_bprop_resid<<<G.J, 256, sm, st>>>(G, D, B, S_L, z);
    // the step index n of the prediction these births belong to is read on the device
    k_bprop_bartlett<<<dim3((Pm.N_g + 7) / 8, Qe), 256, 0, st>>>(G, Pm, D, B);
    k_bprop_moments<<<Qe, 1024, 0, st>>>(Pm, D, B);
    const int nb = (Pm.P + 255) / 256;
    k_bprop_draw<<<nb, 256, 0, st>>>(Pm, D, B, S_L, S_new);
    k_bprop_finish<<<dim3(nb, Qe), 256, 0, st>>>(Pm, D, B, S_L, nb);
    return 6;
}

}  // namespace bp
