// Per-particle update messages (Supplementary Sec. S-V), the hot loop.
//
// Every message is a complex Gaussian whose quadratic form is evaluated in
// its variational (regularised least-squares) form,
//     e^H (eta I + M M^H)^-1 e = min_y |e - M y|^2/eta + |y|^2,
// with the residual r = e - M y* formed element by element.  In this form
// the FP32 error of the result is relative to the residual energy (the
// noise floor) rather than to the signal energy, and errors in y* enter
// only at second order.
//
//  kappa~(phi_s^p, 1)/kappa~(., 0) for every (s, p), summed over j:
//     Delta = J0 - J(tau*) - log(1 + q alpha),
//     J(tau) = |r0 - tau psi_perp|^2/eta_bar + |y0 - tau R^-1 V^H psi/eta_bar|^2 + |tau - a|^2/q,
//     psi_perp = psi - V V^H psi/eta_bar, a = zeta mu^p, q = (gamma^p + |mu^p|^2 (1 - zeta)) zeta,
//     alpha = psi^H A_s^-1 psi, tau* = (psi^H r0/eta_bar + a/q)/(alpha + 1/q).
//  iota~(x^p) for every p, summed over j (columns sqrt(pi (gamma + |mu|^2 (1 - pi))) psi_s):
//     log iota = -|r|^2/eta_bar - |y|^2 - log det(I + D G D/eta_bar) - Nz log(pi eta_bar).
//  nu~(eta^(j,p)) for every (j, p) through the tridiagonal form of G = M^H M.
//
// Steering vectors psi_s^(j,p) = lambda/(4 pi d) e^{-i 2 pi d/lambda} (b kron a_y kron a_z)
// (eq. array-response, unit-modulus-array-response) with d and the local
// direction from FP64 geometry and every phase reduced to cycles in FP64.
#include "bp_internal.cuh"
#include "bp_kernels.cuh"

namespace bp {

// FP32 factors of one steering vector; carrier and amplitude in c.
struct Factors {
    float2 c;
    double A, d;
};

__device__ inline Factors steering_factors(const DevGeom& G, int j, float px, float py, float pz,
                                           float sx, float sy, float sz, bool los,
                                           float2* b, float2* ay, float2* az, int stride) {
    const PathGeo pg = path_geo(G, j, px, py, pz, sx, sy, sz, los);
    Factors F;
    F.d = pg.d;
    F.A = G.lam / (4.0 * M_PI * pg.d);
    double sc, cc;
    sincospi(-2.0 * frac_c(pg.d / G.lam), &sc, &cc);
    F.c = make_float2((float)(F.A * cc), (float)(F.A * sc));
    const double tau = pg.d / G.c;
    for (int f = 0; f < G.Nf; ++f) {
        float s, c;
        sincospif((float)(-2.0 * frac_c(G.f[f] * tau)), &s, &c);
        b[f * stride] = make_float2(c, s);
    }
    const float uy = (float)pg.uy, uz = (float)pg.uz;
    for (int y = 0; y < G.My; ++y) {
        float s, c;
        sincospif(2.0f * (float)(G.py[y] / G.lam) * uy, &s, &c);
        ay[y * stride] = make_float2(c, s);
    }
    for (int m = 0; m < G.Mz; ++m) {
        float s, c;
        sincospif(2.0f * (float)(G.pz[m] / G.lam) * uz, &s, &c);
        az[m * stride] = make_float2(c, s);
    }
    return F;
}

// ---------------------------------------------------------------- kappa
// block = (particle tile of KT threads, s); loop over j; V_{s,j} staged in shared memory.
template <int SC>
__global__ void __launch_bounds__(128) k_kappa(DevGeom G, DevParams Pm, DevState D, int S, int SCA) {
    constexpr int KT = 128;
    constexpr int NC = SC - 1;           // basis columns (zero beyond S-2)
    extern __shared__ float2 sm[];
    const int s = blockIdx.y;
    const int P = Pm.P, J = G.J, Nz = G.Nz, Nm = G.My * G.Mz;
    const int nfac = G.Nf + G.My + G.Mz;
    float2* Vs = sm;                                   // [Nz][SC] (last column r0)
    float2* Rs = Vs + (size_t)Nz * SC;                 // [SC][SC]
    float2* y0s = Rs + (size_t)SC * SC;                // [SC]
    float2* fac = y0s + SC;                            // [nfac][KT]
    const int tid = threadIdx.x;
    const int p = blockIdx.x * KT + tid;
    const bool act = p < P;
    const int pp = act ? p : 0;
    const float* x = D.x[D.cur];
    const float* ph = D.phi[D.cur] + (size_t)s * 6 * P;
    const float px = x[pp], py = x[P + pp], pz = x[2 * P + pp];
    const float sx = ph[pp], sy = ph[P + pp], sz = ph[2 * P + pp];
    const double gm = ph[3 * P + pp];
    const double mr = ph[4 * P + pp], mi = ph[5 * P + pp];
    double delta_sum = 0.0;
    for (int j = 0; j < J; ++j) {
        __syncthreads();
        {   // stage V_{s,j} (first NC columns + r0), R, y0
            const float2* gV = D.kV + ((size_t)s * J + j) * Nz * SCA;
            for (int t = tid; t < Nz * SC; t += KT) {
                const int k = t / SC, c = t - k * SC;
                Vs[t] = (c < NC) ? gV[(size_t)k * SCA + c] : gV[(size_t)k * SCA + SCA - 1];
            }
            const float2* gR = D.kR + ((size_t)s * J + j) * SCA * SCA;
            for (int t = tid; t < SC * SC; t += KT) {
                const int r = t / SC, c = t - r * SC;
                Rs[t] = gR[(size_t)r * SCA + c];
            }
            const float2* gy = D.ky0 + ((size_t)s * J + j) * SCA;
            for (int t = tid; t < SC; t += KT) y0s[t] = gy[t];
        }
        __syncthreads();
        const double eb = D.eta_bar[j];
        const float ebf = (float)eb;
        const double zeta = D.zeta[s * J + j];
        const double J0 = D.kJ0[s * J + j];
        float2* fb = fac + tid;
        float2* fy = fb + G.Nf * KT;
        float2* fz = fy + G.My * KT;
        const Factors F = steering_factors(G, j, px, py, pz, sx, sy, sz, s == 0, fb, fy, fz, KT);
        // pass 1: h = psi^H V, pr = psi^H r0
        float2 h[NC];
        #pragma unroll
        for (int c = 0; c < NC; ++c) h[c] = make_float2(0.f, 0.f);
        float2 pr = make_float2(0.f, 0.f);
        float nps = 0.f;
        for (int f = 0; f < G.Nf; ++f) {
            const float2 cb = cmul(F.c, fb[f * KT]);
            for (int y = 0; y < G.My; ++y) {
                const float2 w = cmul(cb, fy[y * KT]);
                for (int m = 0; m < G.Mz; ++m) {
                    const float2 ps = cmul(w, fz[m * KT]);
                    const int k = f * Nm + y * G.Mz + m;
                    const float2* row = Vs + (size_t)k * SC;
                    #pragma unroll
                    for (int c = 0; c < NC; ++c) {
                        const float2 v = row[c];
                        h[c].x += ps.x * v.x + ps.y * v.y;
                        h[c].y += ps.x * v.y - ps.y * v.x;
                    }
                    const float2 r0 = row[NC];
                    pr.x += ps.x * r0.x + ps.y * r0.y;
                    pr.y += ps.x * r0.y - ps.y * r0.x;
                    nps += ps.x * ps.x + ps.y * ps.y;
                }
            }
        }
        // scalar assembly (FP64)
        double hh = 0.0;
        #pragma unroll
        for (int c = 0; c < NC; ++c) hh += (double)h[c].x * h[c].x + (double)h[c].y * h[c].y;
        const double alpha = ((double)nps - hh / eb) / eb;
        const double2 beta = make_double2(pr.x / eb, pr.y / eb);
        const double2 a = make_double2(zeta * mr, zeta * mi);
        const double q = (gm + (mr * mr + mi * mi) * (1.0 - zeta)) * zeta;
        double2 tau;
        if (q > 0.0) {
            const double den = alpha + 1.0 / q;
            tau = make_double2((beta.x + a.x / q) / den, (beta.y + a.y / q) / den);
        } else {
            tau = a;
        }
        const float2 tf = make_float2((float)tau.x, (float)tau.y);
        // pass 2: r = r0 - tau (psi - V V^H psi / eta_bar), |r|^2
        double rr = 0.0;
        float pn = 0.f;
        for (int f = 0; f < G.Nf; ++f) {
            const float2 cb = cmul(F.c, fb[f * KT]);
            for (int y = 0; y < G.My; ++y) {
                const float2 w = cmul(cb, fy[y * KT]);
                float rr_chunk = 0.f;          // FP32 over the Mz antennas, FP64 across chunks
                for (int m = 0; m < G.Mz; ++m) {
                    const float2 ps = cmul(w, fz[m * KT]);
                    const int k = f * Nm + y * G.Mz + m;
                    const float2* row = Vs + (size_t)k * SC;
                    float2 vv = make_float2(0.f, 0.f);       // V (V^H psi) = sum_c V_kc conj(h_c)
                    #pragma unroll
                    for (int c = 0; c < NC; ++c) {
                        const float2 v = row[c];
                        vv.x += v.x * h[c].x + v.y * h[c].y;
                        vv.y += v.y * h[c].x - v.x * h[c].y;
                    }
                    const float2 pp2 = make_float2(ps.x - vv.x / ebf, ps.y - vv.y / ebf);
                    pn += pp2.x * pp2.x + pp2.y * pp2.y;
                    const float2 r0 = row[NC];
                    const float2 t = cmul(tf, pp2);
                    const float rx = r0.x - t.x, ry = r0.y - t.y;
                    rr_chunk += rx * rx + ry * ry;
                }
                rr += rr_chunk;
            }
        }
        // y = y0 - tau R^-1 V^H psi / eta_bar (back substitution in place: h <- R^-1 conj(h))
        double yy = 0.0, gg = 0.0;
        #pragma unroll
        for (int c = NC - 1; c >= 0; --c) {
            float2 g = make_float2(h[c].x, -h[c].y);
            #pragma unroll
            for (int c2 = c + 1; c2 < NC; ++c2) {
                const float2 u = cmul(Rs[c * SC + c2], h[c2]);
                g.x -= u.x; g.y -= u.y;
            }
            const float dr = Rs[c * SC + c].x;
            h[c] = make_float2(g.x / dr, g.y / dr);
            gg += (double)h[c].x * h[c].x + (double)h[c].y * h[c].y;
            const float2 tg = cmul(tf, h[c]);
            const float2 y0 = y0s[c];
            const double yx = (double)y0.x - (double)tg.x / eb, yi = (double)y0.y - (double)tg.y / eb;
            yy += yx * yx + yi * yi;
        }
        double Jt = rr / eb + yy;
        double logdet = 0.0;
        if (q > 0.0) {
            const double dx = tau.x - a.x, dy = tau.y - a.y;
            Jt += (dx * dx + dy * dy) / q;
            // alpha = psi^H A^-1 psi = |psi_perp|^2/eta_bar + |R^-1 V^H psi|^2/eta_bar^2 (non-negative terms)
            const double alpha_acc = (double)pn / eb + gg / (eb * eb);
            logdet = log1p(q * alpha_acc);
        }
        delta_sum += J0 - Jt - logdet;
    }
    if (act) D.lw_y[(size_t)s * P + p] = delta_sum;
}

// ---------------------------------------------------------------- iota (warp per particle)
// The S x S algebra (Gram of the paired steering vectors, Cholesky, solves) is
// in FP64: the Gram is accumulated from exact FP32 x FP32 products, so that
// log det(eta_bar I + D G D) stays accurate when two columns nearly coincide
// (a FP32 Gram loses 1 - |rho|^2 to rounding).  The residual is FP32.
// per-warp shared memory: factors [S][nfac] (float2), c [S] (double2), c32 [S] (float2),
// d [S] (double), cm [S] (double2), g [S] (double2), A packed lower [S(S+1)/2] (double2)
__device__ inline int tri(int i, int j) { return i * (i + 1) / 2 + j; }

// bytes of one warp's region, rounded up to 16 so that every warp's double2 arrays stay aligned
__host__ __device__ inline size_t iota_warp_bytes(int S, int nfac) {
    const size_t b = (size_t)S * 16 * 3                  // cS, cmS, gS (double2)
                   + (size_t)S * (S + 1) / 2 * 16        // A packed (double2)
                   + (size_t)S * 8                       // dS (double)
                   + (size_t)S * 8                       // c32 (float2)
                   + (size_t)S * nfac * 8;               // factors (float2)
    return (b + 15) / 16 * 16;
}

__global__ void k_iota(DevGeom G, DevParams Pm, DevState D, int S, const float* z) {
    extern __shared__ double2 smd[];
    const int lane = threadIdx.x & 31, wib = threadIdx.x >> 5;
    const int wpb = blockDim.x >> 5;
    const int P = Pm.P, J = G.J, Nz = G.Nz, Nm = G.My * G.Mz;
    const int nfac = G.Nf + G.My + G.Mz;
    float2* zs = reinterpret_cast<float2*>(smd);                               // [Nz]
    char* base = reinterpret_cast<char*>(smd) + (((size_t)Nz * 8 + 15) / 16) * 16 + wib * iota_warp_bytes(S, nfac);
    double2* cS = reinterpret_cast<double2*>(base);                            // [S]
    double2* cmS = cS + S;                                                     // [S]
    double2* gS = cmS + S;                                                     // [S]
    double2* Am = gS + S;                                                      // [S(S+1)/2]
    double* dS = reinterpret_cast<double*>(Am + (size_t)S * (S + 1) / 2);      // [S]
    float2* c32 = reinterpret_cast<float2*>(dS + S);                           // [S]
    float2* fac = c32 + S;                                                     // [S][nfac]
    const int p = blockIdx.x * wpb + wib;
    const bool act = p < P;
    const int pp = act ? p : 0;
    const float* x = D.x[D.cur];
    const float* phi = D.phi[D.cur];
    double total = 0.0;
    for (int j = 0; j < J; ++j) {
        __syncthreads();
        for (int k = threadIdx.x; k < Nz; k += blockDim.x)
            zs[k] = make_float2(z[2 * (j * Nz + k)], z[2 * (j * Nz + k) + 1]);
        __syncthreads();
        const double eb = D.eta_bar[j];
        // 1. factors and coefficients, lanes over s
        for (int s = lane; s < S; s += 32) {
            const float* ph = phi + (size_t)s * 6 * P;
            float2* fs = fac + (size_t)s * nfac;
            const Factors F = steering_factors(G, j, x[pp], x[P + pp], x[2 * P + pp], ph[pp], ph[P + pp], ph[2 * P + pp],
                                               s == 0, fs, fs + G.Nf, fs + G.Nf + G.My, 1);
            double sc, cc;
            sincospi(-2.0 * frac_c(F.d / G.lam), &sc, &cc);
            cS[s] = make_double2(F.A * cc, F.A * sc);
            c32[s] = F.c;
            const double pi = D.zeta[s * J + j] * D.W[s];
            const double gm = ph[3 * P + pp], mr = ph[4 * P + pp], mi = ph[5 * P + pp];
            dS[s] = sqrt(fmax(pi * (gm + (mr * mr + mi * mi) * (1.0 - pi)), 0.0));
            cmS[s] = make_double2(pi * mr, pi * mi);
        }
        __syncwarp();
        // 2. g_s = psi_s^H z (lanes over s, separable contraction, FP32 -> FP64)
        for (int s = lane; s < S; s += 32) {
            const float2* fs = fac + (size_t)s * nfac;
            float2 acc = make_float2(0.f, 0.f);
            for (int f = 0; f < G.Nf; ++f) {
                float2 accy = make_float2(0.f, 0.f);
                for (int y = 0; y < G.My; ++y) {
                    float2 accm = make_float2(0.f, 0.f);
                    for (int m = 0; m < G.Mz; ++m) {
                        const float2 t = cmulc(fs[G.Nf + G.My + m], zs[f * Nm + y * G.Mz + m]);
                        accm.x += t.x; accm.y += t.y;
                    }
                    const float2 t = cmulc(fs[G.Nf + y], accm);
                    accy.x += t.x; accy.y += t.y;
                }
                const float2 t = cmulc(fs[f], accy);
                acc.x += t.x; acc.y += t.y;
            }
            gS[s] = zmulc(cS[s], make_double2(acc.x, acc.y));
        }
        // 3. Gram G_ab = psi_a^H psi_b (a >= b) from the Kronecker factors, FP64 accumulation
        const int npair = S * (S + 1) / 2;
        for (int t = lane; t < npair; t += 32) {
            int a = (int)((sqrtf(8.f * t + 1.f) - 1.f) * 0.5f);
            while ((a + 1) * (a + 2) / 2 <= t) ++a;
            while (a * (a + 1) / 2 > t) --a;
            const int b = t - a * (a + 1) / 2;
            const float2* fa = fac + (size_t)a * nfac;
            const float2* fbb = fac + (size_t)b * nfac;
            double2 sf = make_double2(0, 0), sy = sf, sz = sf;
            for (int f = 0; f < G.Nf; ++f) {
                const double2 u = zmulc(make_double2(fa[f].x, fa[f].y), make_double2(fbb[f].x, fbb[f].y));
                sf.x += u.x; sf.y += u.y;
            }
            for (int y = G.Nf; y < G.Nf + G.My; ++y) {
                const double2 u = zmulc(make_double2(fa[y].x, fa[y].y), make_double2(fbb[y].x, fbb[y].y));
                sy.x += u.x; sy.y += u.y;
            }
            for (int m = G.Nf + G.My; m < nfac; ++m) {
                const double2 u = zmulc(make_double2(fa[m].x, fa[m].y), make_double2(fbb[m].x, fbb[m].y));
                sz.x += u.x; sz.y += u.y;
            }
            Am[t] = zmul(zmulc(cS[a], cS[b]), zmul(sf, zmul(sy, sz)));
        }
        __syncwarp();
        // 4. rhs_a = d_a (g_a - sum_b G_ab cm_b)
        for (int a = lane; a < S; a += 32) {
            double2 acc = gS[a];
            for (int b = 0; b < S; ++b) {
                const double2 gab = (b <= a) ? Am[tri(a, b)] : make_double2(Am[tri(b, a)].x, -Am[tri(b, a)].y);
                const double2 u = zmul(gab, cmS[b]);
                acc.x -= u.x; acc.y -= u.y;
            }
            gS[a] = make_double2(dS[a] * acc.x, dS[a] * acc.y);
        }
        __syncwarp();
        // 5. A = eta_bar I + D G D (packed lower), Cholesky in place
        for (int t = lane; t < npair; t += 32) {
            int a = (int)((sqrtf(8.f * t + 1.f) - 1.f) * 0.5f);
            while ((a + 1) * (a + 2) / 2 <= t) ++a;
            while (a * (a + 1) / 2 > t) --a;
            const int b = t - a * (a + 1) / 2;
            const double dd = dS[a] * dS[b];
            double2 v = Am[t];
            Am[t] = make_double2(dd * v.x + (a == b ? eb : 0.0), dd * v.y);
        }
        __syncwarp();
        double logdet = 0.0;
        for (int k = 0; k < S; ++k) {
            const double dk = sqrt(fmax(Am[tri(k, k)].x, 1e-300));
            logdet += 2.0 * log(dk);
            __syncwarp();
            for (int i = k + 1 + lane; i < S; i += 32) {
                const double2 v = Am[tri(i, k)];
                Am[tri(i, k)] = make_double2(v.x / dk, v.y / dk);
            }
            if (lane == 0) Am[tri(k, k)] = make_double2(dk, 0.0);
            __syncwarp();
            const int n = S - k - 1;
            for (int t = lane; t < n * (n + 1) / 2; t += 32) {
                int a = (int)((sqrtf(8.f * t + 1.f) - 1.f) * 0.5f);
                while ((a + 1) * (a + 2) / 2 <= t) ++a;
                while (a * (a + 1) / 2 > t) --a;
                const int i = k + 1 + a, c = k + 1 + (t - a * (a + 1) / 2);
                const double2 u = zmul(Am[tri(i, k)], make_double2(Am[tri(c, k)].x, -Am[tri(c, k)].y));
                Am[tri(i, c)].x -= u.x; Am[tri(i, c)].y -= u.y;
            }
            __syncwarp();
        }
        // 6. solve L L^H y = rhs
        for (int i = 0; i < S; ++i) {
            double2 acc = make_double2(0, 0);
            for (int b = lane; b < i; b += 32) {
                const double2 u = zmul(Am[tri(i, b)], gS[b]);
                acc.x += u.x; acc.y += u.y;
            }
            acc.x = warp_sum_d(acc.x); acc.y = warp_sum_d(acc.y);
            if (lane == 0) {
                const double dd = Am[tri(i, i)].x;
                gS[i] = make_double2((gS[i].x - acc.x) / dd, (gS[i].y - acc.y) / dd);
            }
            __syncwarp();
        }
        for (int i = S - 1; i >= 0; --i) {
            double2 acc = make_double2(0, 0);
            for (int b = i + 1 + lane; b < S; b += 32) {
                const double2 u = zmulc(Am[tri(b, i)], gS[b]);
                acc.x += u.x; acc.y += u.y;
            }
            acc.x = warp_sum_d(acc.x); acc.y = warp_sum_d(acc.y);
            if (lane == 0) {
                const double dd = Am[tri(i, i)].x;
                gS[i] = make_double2((gS[i].x - acc.x) / dd, (gS[i].y - acc.y) / dd);
            }
            __syncwarp();
        }
        // 7. coefficients w = cm + d y (FP32 copy in c32's slot after use: keep c32, write w into cmS); |y|^2
        double yy = 0.0;
        for (int a = lane; a < S; a += 32) {
            const double2 y = gS[a];
            yy += y.x * y.x + y.y * y.y;
            cmS[a] = make_double2(cmS[a].x + dS[a] * y.x, cmS[a].y + dS[a] * y.y);
        }
        yy = warp_sum_d(yy);
        __syncwarp();
        // 8. residual r = z - sum_s w_s psi_s, element-wise (lanes over elements)
        double rr = 0.0;                   // FP32 per element, FP64 across elements and lanes
        for (int k = lane; k < Nz; k += 32) {
            const int f = k / Nm, ym = k - f * Nm, y = ym / G.Mz, m = ym - y * G.Mz;
            float2 acc = zs[k];
            for (int s = 0; s < S; ++s) {
                const float2* fs = fac + (size_t)s * nfac;
                const float2 ps = cmul(cmul(cmul(c32[s], fs[f]), fs[G.Nf + y]), fs[G.Nf + G.My + m]);
                const float2 u = cmul(make_float2((float)cmS[s].x, (float)cmS[s].y), ps);
                acc.x -= u.x; acc.y -= u.y;
            }
            rr += (double)(acc.x * acc.x + acc.y * acc.y);
        }
        rr = warp_sum_d(rr);
        total += -(rr / eb + yy) - (logdet - S * log(eb)) - Nz * log(M_PI * eb);
    }
    if (act && lane == 0) D.lw_x[p] = total;
}

// ---------------------------------------------------------------- nu (thread per (j, p), FP64)
__global__ void k_nu(DevGeom G, DevParams Pm, DevState D, int S) {
    const int P = Pm.P, SM = Pm.S_max;
    const int idx = blockIdx.x * blockDim.x + threadIdx.x;
    if (idx >= G.J * P) return;
    const int j = idx / P, p = idx - j * P;
    const double eta = (double)D.eta[D.cur][(size_t)j * P + p];
    const double* T = D.nu_T + (size_t)j * 4 * SM;
    double dprev = 1.0, logdet = 0.0, quad = 0.0;
    double ur = 0.0, ui = 0.0;
    double scale = 1.0;
    for (int k = 0; k < S; ++k) {
        double dk = eta + T[k];
        double br = T[2 * SM + 2 * k], bi = T[2 * SM + 2 * k + 1];
        if (k > 0) {
            const double o = T[SM + k - 1];
            const double l = o / dprev;
            dk -= o * l;
            br -= l * ur; bi -= l * ui;
        }
        quad += (br * br + bi * bi) / dk;
        scale *= dk;
        if (scale > 1e200 || scale < 1e-200) { logdet += log(scale); scale = 1.0; }
        dprev = dk; ur = br; ui = bi;
    }
    logdet += log(scale);
    const double e2 = D.nu_c[2 * j];
    const double lnu = -(e2 - quad) / eta - (G.Nz - S) * log(eta) - logdet - G.Nz * log(M_PI);
    D.lw_eta[(size_t)j * P + p] = lnu;
}

template <int SC>
static void launch_kappa_sc(const DevGeom& G, const DevParams& Pm, const DevState& D, int S, int SCA, cudaStream_t st) {
    const int nfac = G.Nf + G.My + G.Mz;
    const size_t smem = ((size_t)G.Nz * SC + (size_t)SC * SC + SC + (size_t)nfac * 128) * sizeof(float2);
    cudaFuncSetAttribute(k_kappa<SC>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    dim3 grid((Pm.P + 127) / 128, S);
    k_kappa<SC><<<grid, 128, smem, st>>>(G, Pm, D, S, SCA);
}

void launch_kappa(const DevGeom& G, const DevParams& Pm, const DevState& D, int S, int SCA, cudaStream_t st) {
    if (S <= 8) launch_kappa_sc<8>(G, Pm, D, S, SCA, st);
    else if (S <= 16) launch_kappa_sc<16>(G, Pm, D, S, SCA, st);
    else if (S <= 32) launch_kappa_sc<32>(G, Pm, D, S, SCA, st);
    else launch_kappa_sc<64>(G, Pm, D, S, SCA, st);
}

size_t kappa_smem_bytes(const DevGeom& G, int S) {
    const int SC = S <= 8 ? 8 : S <= 16 ? 16 : S <= 32 ? 32 : 64;
    const int nfac = G.Nf + G.My + G.Mz;
    return ((size_t)G.Nz * SC + (size_t)SC * SC + SC + (size_t)nfac * 128) * sizeof(float2);
}

void launch_iota(const DevGeom& G, const DevParams& Pm, const DevState& D, int S, const float* z, cudaStream_t st) {
    const int nfac = G.Nf + G.My + G.Mz;
    const size_t per_warp = iota_warp_bytes(S, nfac);
    const size_t zb = (((size_t)G.Nz * 8 + 15) / 16) * 16;
    int wpb = 8;
    while (wpb > 1 && zb + wpb * per_warp > 96 * 1024) wpb /= 2;
    const size_t smem = zb + wpb * per_warp;
    cudaFuncSetAttribute(k_iota, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    k_iota<<<(Pm.P + wpb - 1) / wpb, 32 * wpb, smem, st>>>(G, Pm, D, S, z);
}

void launch_nu(const DevGeom& G, const DevParams& Pm, const DevState& D, int S, cudaStream_t st) {
    const int n = G.J * Pm.P;
    k_nu<<<(n + 255) / 256, 256, 0, st>>>(G, Pm, D, S);
}

}  // namespace bp
