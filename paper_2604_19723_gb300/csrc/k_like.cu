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
//     J(tau) = |r0 - tau psi_perp|^2/eta_bar + |y0 - tau Lambda^-1/2 V^H psi/eta_bar|^2 + |tau - a|^2/q
//     (amplitudes in the eigenbasis of I + M^H M/eta_bar, V its whitened basis),
//     psi_perp = psi - V V^H psi/eta_bar, a = zeta mu^p, q = (gamma^p + |mu^p|^2 (1 - zeta)) zeta,
//     alpha = psi^H A_s^-1 psi, tau* = (psi^H r0/eta_bar + a/q)/(alpha + 1/q).
//  iota~(x^p) for every p, summed over j (columns sqrt(pi (gamma + |mu|^2 (1 - pi))) psi_s):
//     log iota = -|r|^2/eta_bar - |y|^2 - log det(I + D G D/eta_bar) - Nz log(pi eta_bar).
//  nu~(eta^(j,p)) for every (j, p) through the tridiagonal form of G = M^H M.
//
// Steering vectors psi_s^(j,p) = lambda/(4 pi d) e^{-i 2 pi d/lambda} (b kron a_y kron a_z)
// (eq. array-response, unit-modulus-array-response) are rebuilt in FP32 from the
// per-(p, s, j) geometry records of k_geom (FP64 distance and direction).
#include "bp_internal.cuh"
#include "bp_kernels.cuh"
#include "tc_sm100.cuh"

namespace bp {

// ---------------------------------------------------------------- kappa
// block = (particle tile of KT threads, s); loop over j; V_{s,j} staged in shared
// memory as rows of SC complex values (columns 0..SC-2 the eigen-whitened basis,
// column SC-1 the null residual r0), read two columns per 128-bit broadcast load;
// 1/lambda_c and y~0_c = (V^H e0)_c/eta_bar beside it.  The basis columns are orthogonal,
// so every amplitude term is a diagonal sum over the columns.

// The amplitude terms of the PF likelihood in the eigenbasis, with x_c = conj(h_c) =
// (V^H psi)_c, y~0 = V^H e0/eta_bar and v_c = tau x_c/eta_bar:
//     |y0|^2 - |y(tau)|^2 = sum_c (|y~0_c|^2 - |y~0_c - v_c|^2)/lambda_c
//                        = sum_c Re(conj(v_c) (2 y~0_c - v_c))/lambda_c = sum_c g_c.
// Each g_c is small where v_c is, and the sum has no constant of the size of |y~0|^2 to
// cancel.  A column whose terms reach KAPPA_AMP_FF (l (|y~0_c| + |v_c|)^2, l = 1/lambda_c)
// is summed in float-float from exact sums and products of its FP32 operands (a strong
// path, or a PF whose steering vector lies largely in the others' span: FP32 would put
// ~1e-7 of the term on the result, and the term varies from particle to particle); the
// others in FP32, each within ~2e-7 nats.  v_c is rounded to FP32 first: the evaluation
// point then moves by a rounding, which J, minimal there, feels only at second order.
// Also gg = sum_c |h_c|^2/lambda_c, the eigenbasis part of alpha.
// yt: y~0_c, il: 1/lambda_c (.x), u = tau/eta_bar; padded columns have yt = il = 0.
constexpr float KAPPA_AMP_FF = 1.0f;

__device__ __forceinline__ void kappa_amp_ff_term(ff& G, float l, float2 y, float vx, float vy) {
    float ax, axl, ay, ayl;
    two_sum(2.0f * y.x, -vx, ax, axl);   // 2 y~0 - v exactly (2 y~0 is exact)
    two_sum(2.0f * y.y, -vy, ay, ayl);
    const float p1 = __fmul_rn(vx, ax), e1 = fmaf(vx, ax, -p1);
    const float p2 = __fmul_rn(vy, ay), e2 = fmaf(vy, ay, -p2);
    float sh, sl;
    two_sum(p1, p2, sh, sl);
    const float lo = __fadd_rn(__fadd_rn(sl, __fadd_rn(e1, e2)), fmaf(vx, axl, __fmul_rn(vy, ayl)));
    const float q = __fmul_rn(l, sh), eq = fmaf(l, sh, -q);
    float t, et;
    two_sum(G.hi, q, t, et);
    G.hi = t;
    G.lo = __fadd_rn(G.lo, __fadd_rn(et, fmaf(l, lo, eq)));
}

// column c's g_c into G (float-float) or g (FP32), and |h_c|^2/lambda_c into q
__device__ __forceinline__ void kappa_amp_col(ff& G, float& g, float& q, float2 y, float l, float2 hc, float2 u) {
    const float vx = fmaf(u.x, hc.x, u.y * hc.y);     // v = u conj(h)
    const float vy = fmaf(u.y, hc.x, -(u.x * hc.y));
    const float m = fabsf(y.x) + fabsf(y.y) + fabsf(vx) + fabsf(vy);
    if (l * m * m > KAPPA_AMP_FF) kappa_amp_ff_term(G, l, y, vx, vy);
    else g += l * fmaf(vx, fmaf(2.0f, y.x, -vx), vy * fmaf(2.0f, y.y, -vy));
    q = fmaf(l, fmaf(hc.x, hc.x, hc.y * hc.y), q);
}

template <int NC>
__device__ inline void kappa_amp_terms(const float2* yt, const float2* il, const float2 (&h)[NC], float2 u,
                                       double& dyd, float& gg) {
    float g0 = 0.f, g1 = 0.f, q0 = 0.f, q1 = 0.f;
    ff G{0.f, 0.f};
    #pragma unroll
    for (int c = 0; c < NC; ++c) {
        if (c & 1) kappa_amp_col(G, g1, q1, yt[c], il[c].x, h[c], u);
        else       kappa_amp_col(G, g0, q0, yt[c], il[c].x, h[c], u);
    }
    dyd = (double)G.hi + (double)G.lo + (double)(g0 + g1);
    gg = q0 + q1;
}

// MB blocks per SM (register cap 65536 / (256 MB) per thread)
template <int SC, int MB>
__global__ void __launch_bounds__(256, MB) k_kappa(DevGeom G, DevParams Pm, DevState D, int S, int SCA, int fch) {
    constexpr int KT = 256;
    constexpr int NC = SC - 1;           // basis columns (zero beyond S-2)
    constexpr int NP = SC / 2;           // column pairs per row
    extern __shared__ __align__(1024) float4 sm4[];
    const int s = blockIdx.y;
    const int P = Pm.P, J = G.J, Nz = G.Nz, Nm = G.My * G.Mz;
    float4* Vs = sm4;                                                  // [fch * Nm][NP] rows staged
    float2* dls = reinterpret_cast<float2*>(Vs + (size_t)fch * Nm * NP); // [SC] 1/lambda_c (.x)
    float2* y0s = dls + SC;                                            // [SC] y~0_c
    float2* fac = y0s + SC;                                            // [nfac][KT] factors (high parts)
    float2* r0ls = fac + (size_t)(G.Nf + G.My + G.Mz) * KT;           // [fch * Nm] low part of r0
    float2* facl = r0ls + (size_t)fch * Nm;                            // [My + Mz][KT] low parts of a_y, a_z
    // [256] e^{i 2 pi n / 256} as (hi, lo) pairs, on a 16-byte boundary
    float4* ctab = reinterpret_cast<float4*>((reinterpret_cast<uintptr_t>(facl + (size_t)(G.My + G.Mz) * KT) + 15) &
                                             ~(uintptr_t)15);
    float* rn = reinterpret_cast<float*>(ctab + 256);                  // [fch * Nm] |V_k|^2 over the basis columns
    const int tid = threadIdx.x;
    cis_table_fill(ctab, tid, KT);
    const int p = blockIdx.x * KT + tid;
    const bool act = p < P;
    const int pp = act ? p : 0;
    const float* ph = D.phi[D.cur] + (size_t)s * 6 * P;
    const float4* geo_s = D.geo + (size_t)s * J * P;
    const float2* geol_s = D.geo_lo + (size_t)s * J * P;
    const float gmf = ph[3 * P + pp];
    const float mrf = ph[4 * P + pp], mif = ph[5 * P + pp];
    const double mr = mrf, mi = mif;
    double delta_sum = 0.0;
    for (int j = 0; j < J; ++j) {
        const float2* gV = D.kV + ((size_t)s * J + j) * Nz * SCA;
        const float2* gr0l = D.kr0l + ((size_t)s * J + j) * Nz;
        // rows of frequencies [f0, f0 + fch) -> Vs, r0ls (called by all threads)
        auto stage_rows = [&](int f0) {
            float2* Vs2 = reinterpret_cast<float2*>(Vs);
            const int nrow = min(fch, G.Nf - f0) * Nm;
            for (int t = tid; t < nrow * SC; t += KT) {
                const int k = f0 * Nm + t / SC, c = t % SC;
                Vs2[t] = (c < NC) ? gV[(size_t)k * SCA + c] : gV[(size_t)k * SCA + SCA - 1];
            }
            for (int t = tid; t < nrow; t += KT) {
                r0ls[t] = gr0l[f0 * Nm + t];
                const float2* vr = gV + (size_t)(f0 * Nm + t) * SCA;
                float n2 = 0.f;
                for (int c = 0; c < NC; ++c) n2 = fmaf(vr[c].x, vr[c].x, fmaf(vr[c].y, vr[c].y, n2));
                rn[t] = n2;
            }
        };
        __syncthreads();
        {
            if (fch >= G.Nf) stage_rows(0);
            const float2* gd = D.kdl + ((size_t)s * J + j) * SCA;
            const float2* gy = D.ky0 + ((size_t)s * J + j) * SCA;
            for (int t = tid; t < SC; t += KT) { dls[t] = gd[t]; y0s[t] = gy[t]; }
        }
        __syncthreads();
        const double eb = D.eta_bar[j];
        const float ebf = (float)eb;
        const double ieb64 = 1.0 / eb;
        const double zeta = D.zeta[s * J + j];
        const double J0r = D.kJ0[s * J + j];   // |r0|^2 / eta_bar
        float2* fb = fac + tid;
        float2* fy = fb + G.Nf * KT;
        float2* fz = fy + G.My * KT;
        float2* fyl = facl + tid;
        float2* fzl = fyl + G.My * KT;
        // steering factors with the carrier folded into b', evaluated as (hi, lo) pairs; the high
        // parts feed pass 1 (whose rounding only shifts the fitted amplitudes: second order),
        // pass 2 takes the pairs (the low parts of b' are recomputed there per frequency)
        const float4 grec = geo_s[(size_t)j * P + pp];
        const float2 grl = geol_s[(size_t)j * P + pp];
        const float Aamp = G.amp_c / (grec.x + grec.y);
        float ch0, cl0;
        ff_frac_mul2(grec.x, grec.y, G.inv_lam_hi, G.inv_lam_lo, ch0, cl0);
        {
            float2 lo_unused;
            for (int f = 0; f < G.Nf; ++f) bprime_pair(G, ctab, grec.x, grec.y, ch0, cl0, f, fb[f * KT], lo_unused);
            for (int y = 0; y < G.My; ++y) {
                const float p = __fmul_rn(G.py_l[y], grec.z);
                const float e = fmaf(G.py_l[y], grl.x, fmaf(G.py_lo[y], grec.z, fmaf(G.py_l[y], grec.z, -p)));
                cis_pair(ctab, p, e, fy[y * KT], fyl[y * KT]);
            }
            for (int m = 0; m < G.Mz; ++m) {
                const float p = __fmul_rn(G.pz_l[m], grec.w);
                const float e = fmaf(G.pz_l[m], grl.y, fmaf(G.pz_lo[m], grec.w, fmaf(G.pz_l[m], grec.w, -p)));
                cis_pair(ctab, p, e, fz[m * KT], fzl[m * KT]);
            }
        }
        // pass 1: h = psi^H V, pr = psi^H r0
        float2 h[NC];
        #pragma unroll
        for (int c = 0; c < NC; ++c) h[c] = make_float2(0.f, 0.f);
        float2 pr = make_float2(0.f, 0.f);
        float nps = 0.f;
        for (int f0 = 0; f0 < G.Nf; f0 += fch) {
          if (fch < G.Nf) { __syncthreads(); stage_rows(f0); __syncthreads(); }
          for (int f = f0; f < min(G.Nf, f0 + fch); ++f) {
            const float2 cb = make_float2(Aamp * fb[f * KT].x, Aamp * fb[f * KT].y);
            for (int y = 0; y < G.My; ++y) {
                const float2 w = cmul(cb, fy[y * KT]);
                for (int m = 0; m < G.Mz; ++m) {
                    const float2 ps = cmul(w, fz[m * KT]);
                    const float4* row = Vs + (size_t)((f - f0) * Nm + y * G.Mz + m) * NP;
                    #pragma unroll
                    for (int c2 = 0; c2 < NP; ++c2) {
                        // conj(psi) v as explicit FMA chains (4 FMA per complex term)
                        const float4 v = row[c2];
                        h[2 * c2].x = fmaf(ps.x, v.x, fmaf(ps.y, v.y, h[2 * c2].x));
                        h[2 * c2].y = fmaf(ps.x, v.y, fmaf(-ps.y, v.x, h[2 * c2].y));
                        if (2 * c2 + 1 < NC) {
                            h[2 * c2 + 1].x = fmaf(ps.x, v.z, fmaf(ps.y, v.w, h[2 * c2 + 1].x));
                            h[2 * c2 + 1].y = fmaf(ps.x, v.w, fmaf(-ps.y, v.z, h[2 * c2 + 1].y));
                        } else {
                            pr.x = fmaf(ps.x, v.z, fmaf(ps.y, v.w, pr.x));
                            pr.y = fmaf(ps.x, v.w, fmaf(-ps.y, v.z, pr.y));
                        }
                    }
                    nps += ps.x * ps.x + ps.y * ps.y;
                }
            }
          }
        }
        float hh = 0.f;   // alpha here only places tau (the objective is evaluated exactly at it)
        #pragma unroll
        for (int c = 0; c < NC; ++c) hh = fmaf(h[c].x, h[c].x, fmaf(h[c].y, h[c].y, hh));
        // tau in FP32: J is evaluated exactly at the tau used, so its rounding
        // enters Delta at second order only
        const float ieb = 1.0f / ebf;
        const float alpha = (nps - hh * ieb) * ieb;
        // a PF whose steering vector lies mostly in the span of the others' m-vectors (more
        // than 3/4 of its energy) makes psi_perp a small difference: V conj(h) is then summed
        // exactly (products on a grid fixed per element, 2^E > 8 |V_k| |h|), else in FP32 chains
        const bool vh_exact = hh * ieb > 0.75f * nps;
        const float hnorm = sqrtf(hh);
        const float zf = (float)zeta;
        const float2 af = make_float2(zf * mrf, zf * mif);
        const float q = (gmf + (mrf * mrf + mif * mif) * (1.0f - zf)) * zf;
        const float iq = (q > 0.f) ? 1.0f / q : 0.f;
        float2 tf = af;
        if (q > 0.f) {
            const float den = alpha + iq;
            tf = make_float2((pr.x * ieb + af.x * iq) / den, (pr.y * ieb + af.y * iq) / den);
        }
        // pass 2: r = r0 - tau (psi - V V^H psi / eta_bar), |r|^2 and |psi_perp|^2.
        // |r|^2/eta_bar can reach ~1e4 (unmodelled paths), so r is formed in
        // float-float from the exact product tau psi_perp and the two parts of r0,
        // and its squares are summed exactly; V V^H psi runs in eight FP32 chains of
        // an eighth of the columns each, added pairwise.
        ff rr{0.f, 0.f};
        float pn = 0.f;
        for (int f0 = 0; f0 < G.Nf; f0 += fch) {
          if (fch < G.Nf) { __syncthreads(); stage_rows(f0); __syncthreads(); }
          for (int f = f0; f < min(G.Nf, f0 + fch); ++f) {
            // the steering element psi = A b' a_y a_z as a (hi, lo) pair (~1e-9): its error
            // enters the residual at first order
            float2 bh, bl;
            bprime_pair(G, ctab, grec.x, grec.y, ch0, cl0, f, bh, bl);
            const float2 cbh = make_float2(Aamp * bh.x, Aamp * bh.y);
            const float2 cbl = make_float2(fmaf(Aamp, bh.x, -cbh.x) + Aamp * bl.x, fmaf(Aamp, bh.y, -cbh.y) + Aamp * bl.y);
            for (int y = 0; y < G.My; ++y) {
                const float4 wp = cpair_mul(cbh, cbl, fy[y * KT], fyl[y * KT]);
                const float2 wh = make_float2(wp.x, wp.y), wl = make_float2(wp.z, wp.w);
                for (int m = 0; m < G.Mz; ++m) {
                    const float4 psp = cpair_mul(wh, wl, fz[m * KT], fzl[m * KT]);
                    const int kr = (f - f0) * Nm + y * G.Mz + m;
                    const float4* row = Vs + (size_t)kr * NP;
                    constexpr int NCH = NP >= 8 ? 8 : NP;
                    float2 r0 = make_float2(row[NP - 1].z, row[NP - 1].w);
                    float vsx = 0.f, vsy = 0.f, vlx = 0.f, vly = 0.f;   // V conj(h) = (vsx + vlx, vsy + vly)
                    if (vh_exact) {
                        int gE;
                        frexpf(8.0f * sqrtf(rn[kr]) * hnorm + 1e-30f, &gE);
                        const float GM = ldexpf(1.5f, gE);
                        auto grid = [&](float a, float b, float& g, float& q) {
                            const float t = __fsub_rn(fmaf(a, b, GM), GM);
                            g = __fadd_rn(g, t);
                            q += fmaf(a, b, -t);
                        };
                        #pragma unroll
                        for (int c2 = 0; c2 < NP; ++c2) {
                            const float4 v = row[c2];
                            grid(v.x, h[2 * c2].x, vsx, vlx);
                            grid(v.y, h[2 * c2].y, vsx, vlx);
                            grid(v.y, h[2 * c2].x, vsy, vly);
                            grid(-v.x, h[2 * c2].y, vsy, vly);
                            if (2 * c2 + 1 < NC) {
                                grid(v.z, h[2 * c2 + 1].x, vsx, vlx);
                                grid(v.w, h[2 * c2 + 1].y, vsx, vlx);
                                grid(v.w, h[2 * c2 + 1].x, vsy, vly);
                                grid(-v.z, h[2 * c2 + 1].y, vsy, vly);
                            }
                        }
                    } else {
                        float2 va[NCH];
                        #pragma unroll
                        for (int i = 0; i < NCH; ++i) va[i] = make_float2(0.f, 0.f);
                        #pragma unroll
                        for (int c2 = 0; c2 < NP; ++c2) {
                            const int ch = (NCH * c2) / NP;
                            const float4 v = row[c2];
                            va[ch].x = fmaf(v.x, h[2 * c2].x, fmaf(v.y, h[2 * c2].y, va[ch].x));
                            va[ch].y = fmaf(v.y, h[2 * c2].x, fmaf(-v.x, h[2 * c2].y, va[ch].y));
                            if (2 * c2 + 1 < NC) {
                                va[ch].x = fmaf(v.z, h[2 * c2 + 1].x, fmaf(v.w, h[2 * c2 + 1].y, va[ch].x));
                                va[ch].y = fmaf(v.w, h[2 * c2 + 1].x, fmaf(-v.z, h[2 * c2 + 1].y, va[ch].y));
                            }
                        }
                        #pragma unroll
                        for (int w2 = NCH / 2; w2 >= 1; w2 /= 2) {   // pairwise sum of the chains
                            #pragma unroll
                            for (int i = 0; i < w2; ++i) { va[i].x += va[i + w2].x; va[i].y += va[i + w2].y; }
                        }
                        vsx = va[0].x; vsy = va[0].y;
                    }
                    // psi_perp = psi - V V^H psi / eta_bar with the product by 1/eta_bar and the
                    // subtraction taken exactly
                    const float dxh = vsx * ieb, dyh = vsy * ieb;
                    const float dxl = fmaf(vsx, ieb, -dxh) + vlx * ieb, dyl = fmaf(vsy, ieb, -dyh) + vly * ieb;
                    float2 pp2, ppl;
                    two_sum(psp.x, -dxh, pp2.x, ppl.x);
                    two_sum(psp.y, -dyh, pp2.y, ppl.y);
                    ppl.x += psp.z - dxl;
                    ppl.y += psp.w - dyl;
                    pn += pp2.x * pp2.x + pp2.y * pp2.y;
                    // t = tau pp2 exactly: re = p1 - p2, im = p3 + p4 (+ FMA errors)
                    const float p1 = __fmul_rn(tf.x, pp2.x), e1 = fmaf(tf.x, pp2.x, -p1);
                    const float p2 = __fmul_rn(tf.y, pp2.y), e2 = fmaf(tf.y, pp2.y, -p2);
                    const float p3 = __fmul_rn(tf.x, pp2.y), e3 = fmaf(tf.x, pp2.y, -p3);
                    const float p4 = __fmul_rn(tf.y, pp2.x), e4 = fmaf(tf.y, pp2.x, -p4);
                    const float2 rl = r0ls[kr];
                    float sx, ex1, ex2, sy, ey1, ey2;
                    ff rx, ry;
                    two_sum(r0.x, -p1, sx, ex1);
                    two_sum(sx, p2, rx.hi, ex2);
                    rx.lo = __fadd_rn(__fadd_rn(rl.x, __fsub_rn(e2, e1)), __fadd_rn(ex1, ex2));
                    rx.lo = fmaf(-tf.x, ppl.x, fmaf(tf.y, ppl.y, rx.lo));   // - Re(tau psi_perp,lo)
                    two_sum(r0.y, -p3, sy, ey1);
                    two_sum(sy, -p4, ry.hi, ey2);
                    ry.lo = __fsub_rn(__fadd_rn(rl.y, __fadd_rn(ey1, ey2)), __fadd_rn(e3, e4));
                    ry.lo = fmaf(-tf.x, ppl.y, fmaf(-tf.y, ppl.x, ry.lo));  // - Im(tau psi_perp,lo)
                    ff_acc_sq(rr, make_float2(rx.hi, ry.hi));
                    rr.lo = fmaf(2.0f * rx.hi, rx.lo, fmaf(2.0f * ry.hi, ry.lo, rr.lo));
                }
            }
          }
        }
        // amplitude terms in the eigenbasis, column by column (kappa_amp_terms)
        double dyd;
        float gg;
        kappa_amp_terms<NC>(y0s, dls, h, make_float2(tf.x * ieb, tf.y * ieb), dyd, gg);
        double dlt = J0r - ((double)rr.hi + (double)rr.lo) * ieb64 + dyd;
        if (q > 0.f) {
            // prior term |tau - a|^2 / q with the difference taken in FP64 (a may be
            // much larger than the innovation)
            const double dx = (double)tf.x - zeta * mr, dyt = (double)tf.y - zeta * mi;
            dlt -= (dx * dx + dyt * dyt) * (double)iq;
            // alpha = psi^H A^-1 psi = |psi_perp|^2/eta_bar + |R^-1 V^H psi|^2/eta_bar^2 (non-negative terms)
            const float alpha_acc = pn * ieb + gg * ieb * ieb;
            dlt -= (double)log1pf(q * alpha_acc);
        }
        delta_sum += dlt;
    }
    if (act) D.lw_y[(size_t)s * P + p] = delta_sum;
}

// ---------------------------------------------------------------- kappa on the tensor cores
// Both contractions of k_kappa run as tcgen05.mma kind::tf32 in 3xTF32 (hi.hi + hi.lo +
// lo.hi: FP32-level products, FP32 accumulation) with the 128 NT particles of a block as NT
// 128-row M tiles and TMEM accumulators whose lane is the particle.  SW = 64 or 32 basis
// columns (SW - 1 eigen-whitened columns and r0):
//   pass 1, per round of 16 elements: A = psi (Re/Im interleaved), B = rows of
//     [[Re V, Im V], [Im V, -Re V]] -> h = psi^H V (SW - 1 columns) and psi^H r0 in
//     2 SW TMEM columns;
//   pass 2, per group of 32 elements (up to 64 real outputs) and K chunk of 32:
//     A = [Re h, Im h] (from registers), B = rows [[Re V, Im V]; [Im V, -Re V]] over the
//     basis columns (r0 excluded) -> the chunk's part of V conj(h) = V V^H psi for the
//     group's elements, real parts in columns [0, nk), imaginary parts in [nk, 2 nk) of
//     the chunk's own 64-column accumulator.
// Pass 2 is the one contraction whose rounding enters the likelihood at first order, so
// its SW / 16 K chunks accumulate apart (12 MMA accumulations each) and are added pairwise
// in FP32 when the element-wise float-float residual r = r0 - tau (psi - V V^H psi /
// eta_bar) reads them back from TMEM, 8 elements at a time.  Operand tiles of B come
// prebuilt (k_kappa_btile, k_kappa_btile2) by bulk copy; every mbarrier wait is bounded
// (KAPPA_TC_WAIT polls), after which the kernel flags D.kerr, lets copies and MMAs in
// flight land, frees TMEM and ends.
constexpr int KAPPA_TC_WAIT = 1 << 20;
constexpr int KAPPA_TC_KC2 = 32;   // real K per pass-2 chunk (16 basis columns)
constexpr int KAPPA_TC_N2 = 64;    // pass-2 accumulator columns per chunk (SW / 16 chunks x 64 per tile)

// The elements k = f Nm + y Mz + m (Nm = My Mz) are taken in ranges: pass 1 in rounds of
// 16 (KAPPA_TC_KR real K), pass 2 in groups of 32 (up to 64 real outputs).  With
// 2 My Mz in {8, 16, 32} a round is KR / (2 Nm) whole frequencies and a group 32 / Nm;
// with Nm a multiple of 16 a round is part of one frequency.
__host__ __device__ inline int kappa_tc_groups(int Nf, int Nm) { return (Nf * Nm + 31) / 32; }
__host__ __device__ inline int round16(int x) { return (x + 15) & ~15; }
// Pass 1's two accumulators alternate by round; every KAPPA_TC_SEG rounds of one (five
// when a round is one frequency of the 4 x 4 URA, as validated at full size; else two,
// i.e. 24 MMA accumulations, the chain that stayed within 1e-4) it is added into
// registers and restarted.  Above KAPPA_TC_FLY_NF frequencies the frequency factors are
// formed when used instead of being kept in shared memory.
constexpr int KAPPA_TC_KR = 32;
constexpr int KAPPA_TC_FLY_NF = 16;
__host__ __device__ inline int kappa_tc_f1(int Nm) { return KAPPA_TC_KR / (2 * Nm); }   // 0 when Nm > 16
__host__ __device__ inline int kappa_tc_r1(int Nf, int Nm) { return (Nf * Nm + 15) / 16; }
__host__ __device__ inline int kappa_tc_seg(int Nm) { return 2 * Nm == KAPPA_TC_KR ? 5 : 2; }
// operand region in floats for SW basis columns (incl. r0): pass 1 A [NT][hi, lo][128 x KR]
// and one B slot [hi, lo][2 SW x KR]; pass 2 A [NT][hi, lo][128 x KC2] and two B slots
// [hi, lo][64 x KC2]
__host__ __device__ inline int kappa_tc_region_floats(int SW, int NT) {
    const int r1 = 2 * NT * 128 * KAPPA_TC_KR + 2 * (2 * SW) * KAPPA_TC_KR;
    const int r2 = 2 * NT * 128 * KAPPA_TC_KC2 + 2 * 2 * KAPPA_TC_N2 * KAPPA_TC_KC2;
    return r1 > r2 ? r1 : r2;
}

// NT 128-particle M tiles per block (threads 128 NT, TMEM columns 256 NT): NT = 1 lets two
// blocks share an SM, so that one block's MMAs run while the other writes operands or
// evaluates its residuals.
// LARGE: the arrays of My Mz >= 32 elements (a multiple of 16): pass-1 rounds within one
// frequency, and pass 2 forms psi as a (hi, lo) pair (~1e-9) from factors evaluated by
// cis_pair, with psi - V conj(h) / eta_bar taken exactly; at Nz = 1024 and 30 dB the FP32
// steering values' few ulps, which enter the residual at first order, put 1.2e-4 on the PF
// weights.  Its frequency factors are formed when used.
template <int NT, int SW, bool LARGE>
__global__ void __launch_bounds__(128 * NT, NT == 1 ? 2 : 1) k_kappa_tc(DevGeom G, DevParams Pm, DevState D, int S, int SCA,
                                                                     const float* __restrict__ Bt1,
                                                                     const float* __restrict__ Bt2) {
    static_assert(SW == 64 || SW == 32, "basis width");
    static_assert(SW == 64 || LARGE, "32 columns only for the large arrays");
    constexpr int KT = 128 * NT, NC = SW - 1, KC2 = KAPPA_TC_KC2;
    constexpr int N1 = 2 * SW;                                 // pass-1 accumulator columns
    constexpr int NCH = SW / 16;                               // pass-2 K chunks
    extern __shared__ __align__(1024) float4 sm4[];
    const int s = blockIdx.y;
    const int P = Pm.P, J = G.J, Nz = G.Nz, Nm = G.My * G.Mz, Nf = G.Nf;
    const int KC = 2 * Nm;                                     // pass-1 real K per frequency
    constexpr int KR = KAPPA_TC_KR;                            // pass-1 real K per round
    const int F1 = kappa_tc_f1(Nm), R1 = kappa_tc_r1(Nf, Nm), SEG = kappa_tc_seg(Nm);
    const bool fly = LARGE || Nf > KAPPA_TC_FLY_NF;            // frequency factors formed when used
    const int NG = kappa_tc_groups(Nf, Nm);
    const int RF = kappa_tc_region_floats(SW, NT);            // operand region (floats)
    float* sR = reinterpret_cast<float*>(sm4);
    uint64_t* mbar = reinterpret_cast<uint64_t*>(sR + RF);    // [3]: MMAs done, B slot 0, B slot 1 arrived
    uint32_t* tslot = reinterpret_cast<uint32_t*>(mbar + 3);
    float4* r0s = reinterpret_cast<float4*>(sR + RF + 8);    // [Nz] r0 (hi.x, hi.y, lo.x, lo.y)
    float2* dls = reinterpret_cast<float2*>(r0s + Nz);        // [SW] 1/lambda_c (.x)
    float2* y0s = dls + SW;                                   // [SW] y~0_c
    float2* fac = y0s + SW;                                   // [nfac][KT]
    // LARGE: [Mz][KT] low parts of a_z, then the (hi, lo) cis table [256] on a 16-byte boundary
    float2* facl = fac + (size_t)((fly ? 0 : Nf) + G.My + G.Mz) * KT;
    float4* ctab = reinterpret_cast<float4*>((reinterpret_cast<uintptr_t>(facl + (size_t)G.Mz * KT) + 15) &
                                             ~(uintptr_t)15);
    const int tid = threadIdx.x, warp = tid >> 5, tile = tid >> 7, row = tid & 127;
    if (LARGE) cis_table_fill(ctab, tid, KT);   // read after the first barrier of the j loop
    const int p = blockIdx.x * KT + tid;
    const bool act = p < P;
    const int pp = act ? p : 0;
    const uint32_t mb_mma = tc::smem_u32(&mbar[0]), mb_b0 = tc::smem_u32(&mbar[1]);   // slot sl: mb_b0 + 8 sl
    uint32_t n_commit = 0;
    uint32_t b_pend = 0, b_par = 0;   // thread 0: per B slot, a copy in flight / the parity of its next wait
    bool bad = false;
    if (warp == 0) tc::tmem_alloc(tslot, 256 * NT);
    if (tid == 0) { tc::mbar_init(mb_mma, 1); tc::mbar_init(mb_b0, 1); tc::mbar_init(mb_b0 + 8, 1); tc::mbar_init_fence(); }
    tc::fence_before_sync();
    __syncthreads();
    tc::fence_after_sync();
    // B operand stream (thread 0): pass 1 takes one slot of 2 x N1 x KR floats at
    // sR + 2 NT 128 KR; pass 2 two slots of 2 x 64 x KC2 floats after its A tiles, so that
    // the copy of the next round's B runs under this round's MMAs.  A copy into a slot is
    // issued only once the MMAs that read the slot's previous contents have completed.
    const size_t bchunk1 = (size_t)2 * N1 * KR;
    const size_t bslot2 = (size_t)2 * KAPPA_TC_N2 * KC2;
    const int NQ = NCH * NG;   // pass-2 rounds per j
    float* sB1 = sR + 2 * NT * 128 * KR;
    float* sB2 = sR + 2 * NT * 128 * KC2;
    auto issueB = [&](int sl, float* dst, const float* src, uint32_t bytes) {
        if (tid != 0 || bad) return;
        const uint32_t mb = mb_b0 + 8u * (uint32_t)sl;
        tc::mbar_expect_tx(mb, bytes);
        tc::bulk_g2s(tc::smem_u32(dst), src, bytes, mb);
        b_pend |= 1u << sl;
    };
    auto waitB = [&](int sl) -> bool {   // thread 0
        const uint32_t mb = mb_b0 + 8u * (uint32_t)sl;
        if (!tc::mbar_wait(mb, (b_par >> sl) & 1u, KAPPA_TC_WAIT)) return false;
        b_par ^= 1u << sl;
        b_pend &= ~(1u << sl);
        return true;
    };
    auto b1_src = [&](int j, int r) { return Bt1 + (((size_t)s * J + j) * R1 + r) * bchunk1; };
    auto b2_src = [&](int j, int q) { return Bt2 + (((size_t)s * J + j) * NQ + q) * bslot2; };
    auto b2_bytes = [&](int q) {
        const int g = q / NCH, nk = min(32, Nz - 32 * g);
        return (uint32_t)(2 * (2 * round16(nk)) * KC2 * 4);
    };
    issueB(0, sB1, b1_src(0, 0), (uint32_t)(bchunk1 * 4));   // the first round's B, under the factor set-up
    const uint32_t tmem = *tslot;
    const uint32_t tlane = tmem + ((uint32_t)((warp & 3) * 32) << 16) + (uint32_t)(tile * 256);   // this thread's row
    const float* ph = D.phi[D.cur] + (size_t)s * 6 * P;
    const float4* geo_s = D.geo + (size_t)s * J * P;
    const float2* geol_s = D.geo_lo + (size_t)s * J * P;
    const float gmf = ph[3 * P + pp];
    const float mrf = ph[4 * P + pp], mif = ph[5 * P + pp];
    const double mr = mrf, mi = mif;
    // one round: once the previous round's MMAs are done, issueNext() starts a B copy
    // (thread 0) and every thread writes A (writeA); after the barrier thread 0 waits for
    // this round's B (slot sl) and issues the 3xTF32 MMAs of both tiles (K in steps of 8)
    auto round = [&](int sl, float* sA, float* sB, int Kt, uint32_t bLoOff, uint32_t idesc, uint32_t dcol,
                     bool accum0, auto&& issueNext, auto&& writeA) {
        if (n_commit > 0 && !bad && !tc::mbar_wait(mb_mma, (n_commit - 1) & 1u, KAPPA_TC_WAIT)) bad = true;
        issueNext();
        writeA();
        tc::fence_async_smem();
        tc::fence_before_sync();
        __syncthreads();
        tc::fence_after_sync();
        if (tid == 0 && !bad) {
            if (!waitB(sl)) bad = true;
            if (!bad) {
                const uint32_t sbo = (uint32_t)(Kt / 4) * 128u;
                const uint32_t bH = tc::smem_u32(sB), bL = bH + bLoOff;
                for (int t = 0; t < NT; ++t) {
                    const uint32_t aH = tc::smem_u32(sA + (size_t)(t * 2) * 128 * Kt);
                    const uint32_t aL = tc::smem_u32(sA + (size_t)(t * 2 + 1) * 128 * Kt);
                    for (int ks = 0; ks < Kt / 8; ++ks) {
                        const uint32_t o = (uint32_t)ks * 256u;
                        const uint64_t dAH = tc::smem_desc(aH + o, 128, sbo), dAL = tc::smem_desc(aL + o, 128, sbo);
                        const uint64_t dBH = tc::smem_desc(bH + o, 128, sbo), dBL = tc::smem_desc(bL + o, 128, sbo);
                        const uint32_t d = tmem + (uint32_t)(t * 256) + dcol;
                        tc::mma_tf32(d, dAH, dBH, idesc, accum0 || ks > 0);
                        tc::mma_tf32(d, dAH, dBL, idesc, true);
                        tc::mma_tf32(d, dAL, dBH, idesc, true);
                    }
                }
                tc::mma_commit(mb_mma);
            }
        }
        ++n_commit;
    };
    auto wait_mma = [&]() {
        if (!bad && !tc::mbar_wait(mb_mma, (n_commit - 1) & 1u, KAPPA_TC_WAIT)) bad = true;
        tc::fence_after_sync();
    };
    double delta_sum = 0.0;
    for (int j = 0; j < J; ++j) {
        const float2* gV = D.kV + ((size_t)s * J + j) * Nz * SCA;
        const float2* gr0l = D.kr0l + ((size_t)s * J + j) * Nz;
        __syncthreads();
        for (int k = tid; k < Nz; k += KT) {
            const float2 hi = gV[(size_t)k * SCA + SCA - 1], lo = gr0l[k];
            r0s[k] = make_float4(hi.x, hi.y, lo.x, lo.y);
        }
        {
            const float2* gd = D.kdl + ((size_t)s * J + j) * SCA;
            const float2* gy = D.ky0 + ((size_t)s * J + j) * SCA;
            for (int t = tid; t < SW; t += KT) { dls[t] = gd[t]; y0s[t] = gy[t]; }
        }
        __syncthreads();
        const double eb = D.eta_bar[j];
        const float ebf = (float)eb;
        const double ieb64 = 1.0 / eb;
        const double zeta = D.zeta[s * J + j];
        const double J0r = D.kJ0[s * J + j];
        float2* fb = fac + tid;                                // [Nf][KT] unless fly
        float2* fy = fb + (fly ? 0 : Nf) * KT;
        float2* fz = fy + G.My * KT;
        const float4 grec = geo_s[(size_t)j * P + pp];
        const float2 grl = geol_s[(size_t)j * P + pp];
        float2 Fc;
        float Aamp = 0.f, ch0 = 0.f, cl0 = 0.f;   // LARGE: psi = A (b' kron a_y kron a_z), carrier in b'
        float2* fzl = facl + tid;
        // the phase of a_y (cycles, float-float) and its (hi, lo) pair
        auto ay_phase = [&](int y, float& p, float& e) {
            p = __fmul_rn(G.py_l[y], grec.z);
            e = fmaf(G.py_l[y], grl.x, fmaf(G.py_lo[y], grec.z, fmaf(G.py_l[y], grec.z, -p)));
        };
        if (LARGE) {
            Aamp = G.amp_c / (grec.x + grec.y);
            ff_frac_mul2(grec.x, grec.y, G.inv_lam_hi, G.inv_lam_lo, ch0, cl0);
            Fc = make_float2(Aamp, 0.f);   // cmul(Fc, b') = A b' exactly
            float2 lo_unused;
            for (int y = 0; y < G.My; ++y) {
                float p, e;
                ay_phase(y, p, e);
                cis_pair(ctab, p, e, fy[y * KT], lo_unused);
            }
            for (int m = 0; m < G.Mz; ++m) {
                const float p = __fmul_rn(G.pz_l[m], grec.w);
                const float e = fmaf(G.pz_l[m], grl.y, fmaf(G.pz_lo[m], grec.w, fmaf(G.pz_l[m], grec.w, -p)));
                cis_pair(ctab, p, e, fz[m * KT], fzl[m * KT]);
            }
        } else if (fly) {
            Fc = carrier_factor(G, grec);
            array_factors(G, grec, grl, fy, fz, KT);
        } else {
            Fc = factors_from_geo(G, grec, grl, fb, fy, fz, KT);
        }
        // b_f as pass 1 and pass 2 both take it (the shared copy holds the same values);
        // LARGE: the high part of b'_f
        auto bfac = [&](int f) {
            if (LARGE) {
                float2 bh, bl;
                bprime_pair(G, ctab, grec.x, grec.y, ch0, cl0, f, bh, bl);
                return bh;
            }
            return fly ? freq_factor(G, grec, f) : fb[f * KT];
        };
        // h = psi^H V and pr = psi^H r0, summed over the pass-1 accumulator segments
        float2 h[NC];
        float2 pr = make_float2(0.f, 0.f);
        #pragma unroll
        for (int c = 0; c < NC; ++c) h[c] = make_float2(0.f, 0.f);
        // adds the pass-1 accumulator at TMEM column base (N1 columns: Re h 0..NC-1, Re pr,
        // Im h 0..NC-1, Im pr) into h and pr, 32 columns at a time
        auto absorb = [&](uint32_t base) {
            #pragma unroll
            for (int part = 0; part < 2; ++part) {
                #pragma unroll
                for (int c0 = 0; c0 < SW; c0 += 32) {
                    uint32_t v[32];
                    tc::tmem_ld32(tlane + base + (uint32_t)(part * SW + c0), v);
                    tc::tmem_ld_wait();
                    #pragma unroll
                    for (int i = 0; i < 32; ++i) {
                        const float a = __uint_as_float(v[i]);
                        if (c0 + i < NC) { if (part == 0) h[c0 + i].x += a; else h[c0 + i].y += a; }
                        else             { if (part == 0) pr.x += a; else pr.y += a; }
                    }
                }
            }
        };
        // ---- pass 1: h = psi^H V, pr = psi^H r0, 16 elements per round
        float nps = 0.f;
        {
            float* sA = sR;
            float* aHi = sA + (size_t)(tile * 2 + 0) * 128 * KR;
            float* aLo = sA + (size_t)(tile * 2 + 1) * 128 * KR;
            const uint32_t idesc = tc::idesc_tf32_f32(128, N1);
            // even rounds accumulate in columns 0..N1-1, odd ones in N1..2 N1-1; a segment of
            // SEG rounds of one accumulator is added into h (after the MMAs of the previous
            // round are done, before this round overwrites it); the first round's B was
            // issued before this j began
            for (int r = 0; r < R1; ++r) {
                const int q = r & 1;
                const bool seg_start = ((r >> 1) % SEG) == 0;
                round(0, sA, sB1, KR, (uint32_t)(N1 * KR * 4), idesc, (uint32_t)(q * N1), !seg_start,
                      [&]() {
                    if (seg_start && r >= 2) absorb((uint32_t)(q * N1));
                    if (r > 0) issueB(0, sB1, b1_src(j, r), (uint32_t)(bchunk1 * 4));
                }, [&]() {
                    if constexpr (LARGE) {
                        // Nm a multiple of 16: the round is elements 16 r .. 16 r + 15 of one
                        // frequency, walked in pairs (m, m + 1) of a row (Mz even)
                        const int k0 = r * 16, f = k0 / Nm, e0 = k0 - f * Nm;
                        const float2 cb = cmul(Fc, bfac(f));
                        int y = e0 / G.Mz, m = e0 - y * G.Mz;
                        float2 w = cmul(cb, fy[y * KT]);
                        #pragma unroll 1
                        for (int l = 0; l < 16; l += 2) {
                            const float2 p0 = cmul(w, fz[m * KT]), p1 = cmul(w, fz[(m + 1) * KT]);
                            nps += p0.x * p0.x + p0.y * p0.y + p1.x * p1.x + p1.y * p1.y;
                            const float4 hi = make_float4(tc::tf32_rn(p0.x), tc::tf32_rn(p0.y), tc::tf32_rn(p1.x),
                                                          tc::tf32_rn(p1.y));
                            const float4 lo = make_float4(tc::tf32_rn(p0.x - hi.x), tc::tf32_rn(p0.y - hi.y),
                                                          tc::tf32_rn(p1.x - hi.z), tc::tf32_rn(p1.y - hi.w));
                            const int off = tc::core_off(row, 2 * l, KR) >> 2;
                            *reinterpret_cast<float4*>(aHi + off) = hi;
                            *reinterpret_cast<float4*>(aLo + off) = lo;
                            m += 2;
                            if (m == G.Mz && l + 2 < 16) { m = 0; ++y; w = cmul(cb, fy[y * KT]); }
                        }
                    } else {
                    for (int i = 0; i < F1; ++i) {
                        const int f = r * F1 + i;
                        if (f >= Nf) {   // past the last frequency: zero operands
                            for (int kk = i * KC; kk < (i + 1) * KC; kk += 4) {
                                const int off = tc::core_off(row, kk, KR) >> 2;
                                *reinterpret_cast<float4*>(aHi + off) = make_float4(0.f, 0.f, 0.f, 0.f);
                                *reinterpret_cast<float4*>(aLo + off) = make_float4(0.f, 0.f, 0.f, 0.f);
                            }
                            continue;
                        }
                        const float2 cb = cmul(Fc, bfac(f));
                        for (int y = 0; y < G.My; ++y) {
                            const float2 w = cmul(cb, fy[y * KT]);
                            for (int m = 0; m < G.Mz; m += 2) {
                                const float2 p0 = cmul(w, fz[m * KT]), p1 = cmul(w, fz[(m + 1) * KT]);
                                nps += p0.x * p0.x + p0.y * p0.y + p1.x * p1.x + p1.y * p1.y;
                                const float4 hi = make_float4(tc::tf32_rn(p0.x), tc::tf32_rn(p0.y), tc::tf32_rn(p1.x),
                                                              tc::tf32_rn(p1.y));
                                const float4 lo = make_float4(tc::tf32_rn(p0.x - hi.x), tc::tf32_rn(p0.y - hi.y),
                                                              tc::tf32_rn(p1.x - hi.z), tc::tf32_rn(p1.y - hi.w));
                                const int off = tc::core_off(row, i * KC + 2 * (y * G.Mz + m), KR) >> 2;
                                *reinterpret_cast<float4*>(aHi + off) = hi;
                                *reinterpret_cast<float4*>(aLo + off) = lo;
                            }
                        }
                    }
                    }
                });
            }
        }
        wait_mma();
        // pass 2's first two B tiles, under the read-back of h and the amplitude sums
        issueB(0, sB2, b2_src(j, 0), b2_bytes(0));
        issueB(1, sB2 + bslot2, b2_src(j, 1), b2_bytes(1));
        absorb(0);                       // the segments still in TMEM
        if (R1 > 1) absorb((uint32_t)N1);
        // h and pr back into columns 0..N1-1 (the accumulator layout), where the amplitude
        // loop reads them
        #pragma unroll
        for (int part = 0; part < 2; ++part) {
            #pragma unroll
            for (int c0 = 0; c0 < SW; c0 += 32) {
                uint32_t v[32];
                #pragma unroll
                for (int i = 0; i < 32; ++i) {
                    const float2 a = (c0 + i < NC) ? h[c0 + i] : pr;
                    v[i] = __float_as_uint(part == 0 ? a.x : a.y);
                }
                tc::tmem_st32(tlane + (uint32_t)(part * SW + c0), v);
            }
        }
        tc::tmem_st_wait();
        // tau (FP32; J is evaluated exactly at the tau used) and the O(S) amplitude sums
        float hh = 0.f;
        #pragma unroll
        for (int c = 0; c < NC; ++c) hh = fmaf(h[c].x, h[c].x, fmaf(h[c].y, h[c].y, hh));
        const float ieb = 1.0f / ebf;
        const float alpha = (nps - hh * ieb) * ieb;
        const float zf = (float)zeta;
        const float2 af = make_float2(zf * mrf, zf * mif);
        const float q = (gmf + (mrf * mrf + mif * mif) * (1.0f - zf)) * zf;
        const float iq = (q > 0.f) ? 1.0f / q : 0.f;
        float2 tf = af;
        if (q > 0.f) {
            const float den = alpha + iq;
            tf = make_float2((pr.x * ieb + af.x * iq) / den, (pr.y * ieb + af.y * iq) / den);
        }
        // amplitude terms in the eigenbasis (kappa_amp_terms), h read again from TMEM columns
        // 0..N1-1 (written back above) eight columns at a time: a rolled loop keeps the
        // per-column code out of the instruction cache's way
        double dyd;
        float gg;
        {
            const float2 u = make_float2(tf.x * ieb, tf.y * ieb);
            float g0 = 0.f, g1 = 0.f, q0 = 0.f, q1 = 0.f;
            ff G{0.f, 0.f};
            #pragma unroll 1
            for (int c0 = 0; c0 < SW; c0 += 8) {
                uint32_t a[8], b[8];
                float hx[8], hy[8];
                tc::tmem_ld8(tlane + (uint32_t)c0, a);
                tc::tmem_ld8(tlane + (uint32_t)(SW + c0), b);
                tc::tmem_ld_wait();
                #pragma unroll
                for (int i = 0; i < 8; ++i) { hx[i] = __uint_as_float(a[i]); hy[i] = __uint_as_float(b[i]); }
                #pragma unroll
                for (int i = 0; i < 8; ++i) {
                    const int c = c0 + i;
                    if (c < NC) {   // column NC holds psi^H r0
                        if (i & 1) kappa_amp_col(G, g1, q1, y0s[c], dls[c].x, make_float2(hx[i], hy[i]), u);
                        else       kappa_amp_col(G, g0, q0, y0s[c], dls[c].x, make_float2(hx[i], hy[i]), u);
                    }
                }
            }
            dyd = (double)G.hi + (double)G.lo + (double)(g0 + g1);
            gg = q0 + q1;
        }
        // ---- pass 2: V V^H psi per group of frequencies, then the element-wise residual
        ff rr{0.f, 0.f};
        float pn = 0.f;
        tc::fence_before_sync();   // TMEM reads of h complete before pass 2 reuses the columns
        for (int g = 0; g < NG; ++g) {
            const int k0 = 32 * g, nk = min(32, Nz - k0), nkp = round16(nk), N2 = 2 * nkp;
            float* sA = sR;
            float* aHi = sA + (size_t)(tile * 2 + 0) * 128 * KC2;
            float* aLo = sA + (size_t)(tile * 2 + 1) * 128 * KC2;
            const uint32_t idesc = tc::idesc_tf32_f32(128, N2);
            #pragma unroll
            for (int kc = 0; kc < NCH; ++kc) {
                // round q = NCH g + kc reads slot q & 1 = kc & 1 (NCH is even); the copy of
                // round q + 1 goes to the slot that round q - 1 read
                const int q = NCH * g + kc;
                round(kc & 1, sA, sB2 + (size_t)(kc & 1) * bslot2, KC2, (uint32_t)(N2 * KC2 * 4), idesc,
                      (uint32_t)(kc * KAPPA_TC_N2), false, [&]() {
                    if (q >= 1 && q + 1 < NQ)
                        issueB((q + 1) & 1, sB2 + (size_t)((q + 1) & 1) * bslot2, b2_src(j, q + 1), b2_bytes(q + 1));
                }, [&]() {
                    #pragma unroll
                    for (int c2 = 0; c2 < KC2 / 4; ++c2) {       // basis columns c, c + 1
                        const int c = kc * 16 + 2 * c2;
                        const float2 u0 = h[c];
                        const float2 u1 = (c + 1 < NC) ? h[c + 1] : make_float2(0.f, 0.f);
                        const float4 hi = make_float4(tc::tf32_rn(u0.x), tc::tf32_rn(u0.y), tc::tf32_rn(u1.x), tc::tf32_rn(u1.y));
                        const float4 lo = make_float4(tc::tf32_rn(u0.x - hi.x), tc::tf32_rn(u0.y - hi.y),
                                                      tc::tf32_rn(u1.x - hi.z), tc::tf32_rn(u1.y - hi.w));
                        const int off = tc::core_off(row, 4 * c2, KC2) >> 2;
                        *reinterpret_cast<float4*>(aHi + off) = hi;
                        *reinterpret_cast<float4*>(aLo + off) = lo;
                    }
                });
            }
            wait_mma();
            // every MMA of this j is done: the next j's first B tile, under the residuals
            if (g == NG - 1 && j + 1 < J) issueB(0, sB1, b1_src(j + 1, 0), (uint32_t)(bchunk1 * 4));
            // element (f, y, m) of the group walked in order from k0; w = Fc b_f a_y formed as
            // pass 1 formed it (LARGE: the pair (wh, wl) = A b'_f a_y from cis_pair factors)
            int cf = k0 / Nm, cy = (k0 - cf * Nm) / G.Mz, cm = k0 - cf * Nm - cy * G.Mz;
            float2 w = make_float2(0.f, 0.f), wh = w, wl = w;
            auto set_w = [&]() {
                if (LARGE) {
                    float2 bh, bl, ayh, ayl;
                    bprime_pair(G, ctab, grec.x, grec.y, ch0, cl0, cf, bh, bl);
                    const float2 cbh = make_float2(Aamp * bh.x, Aamp * bh.y);
                    const float2 cbl = make_float2(fmaf(Aamp, bh.x, -cbh.x) + Aamp * bl.x,
                                                   fmaf(Aamp, bh.y, -cbh.y) + Aamp * bl.y);
                    float p, e;
                    ay_phase(cy, p, e);
                    cis_pair(ctab, p, e, ayh, ayl);
                    const float4 wp = cpair_mul(cbh, cbl, ayh, ayl);
                    wh = make_float2(wp.x, wp.y);
                    wl = make_float2(wp.z, wp.w);
                } else {
                    w = cmul(cmul(Fc, bfac(cf)), fy[cy * KT]);
                }
            };
            set_w();
            for (int b = 0; b < nk; b += 8) {
                // the chunk accumulators, added pairwise: (a0 + a1) [+ (a2 + a3)]
                float vre[8], vim[8];
                #pragma unroll
                for (int c2 = 0; c2 < NCH; c2 += 2) {
                    uint32_t r0[8], r1[8], i0[8], i1[8];
                    tc::tmem_ld8(tlane + (uint32_t)(c2 * KAPPA_TC_N2 + b), r0);
                    tc::tmem_ld8(tlane + (uint32_t)((c2 + 1) * KAPPA_TC_N2 + b), r1);
                    tc::tmem_ld8(tlane + (uint32_t)(c2 * KAPPA_TC_N2 + nkp + b), i0);
                    tc::tmem_ld8(tlane + (uint32_t)((c2 + 1) * KAPPA_TC_N2 + nkp + b), i1);
                    tc::tmem_ld_wait();
                    #pragma unroll
                    for (int i = 0; i < 8; ++i) {
                        const float ar = __uint_as_float(r0[i]) + __uint_as_float(r1[i]);
                        const float ai = __uint_as_float(i0[i]) + __uint_as_float(i1[i]);
                        if (c2 == 0) { vre[i] = ar; vim[i] = ai; }
                        else         { vre[i] += ar; vim[i] += ai; }
                    }
                }
                #pragma unroll
                for (int i = 0; i < 8; ++i) {
                    const int kl = b + i;
                    if (kl >= nk) break;
                    const int k = k0 + kl;
                    float2 ps;         // psi_k exactly as pass 1 formed it
                    float4 psp;        // LARGE: psi_k as a (hi, lo) pair
                    if (LARGE) psp = cpair_mul(wh, wl, fz[cm * KT], fzl[cm * KT]);
                    else       ps = cmul(w, fz[cm * KT]);
                    if (++cm == G.Mz) {
                        cm = 0;
                        if (++cy == G.My) { cy = 0; ++cf; }
                        if (kl + 1 < nk) set_w();
                    }
                    const float vsx = vre[i], vsy = vim[i];
                    float2 pp2, ppl = make_float2(0.f, 0.f);
                    if (LARGE) {
                        // psi_perp = psi - V V^H psi / eta_bar with the product by 1/eta_bar and
                        // the subtraction taken exactly; its low part ppl
                        const float dxh = vsx * ieb, dyh = vsy * ieb;
                        const float dxl = fmaf(vsx, ieb, -dxh), dyl = fmaf(vsy, ieb, -dyh);
                        two_sum(psp.x, -dxh, pp2.x, ppl.x);
                        two_sum(psp.y, -dyh, pp2.y, ppl.y);
                        ppl.x += psp.z - dxl;
                        ppl.y += psp.w - dyl;
                    } else {
                        pp2 = make_float2(ps.x - vsx * ieb, ps.y - vsy * ieb);
                    }
                    pn += pp2.x * pp2.x + pp2.y * pp2.y;
                    // t = tau pp2 exactly: re = p1 - p2, im = p3 + p4 (+ FMA errors)
                    const float p1 = __fmul_rn(tf.x, pp2.x), e1 = fmaf(tf.x, pp2.x, -p1);
                    const float p2 = __fmul_rn(tf.y, pp2.y), e2 = fmaf(tf.y, pp2.y, -p2);
                    const float p3 = __fmul_rn(tf.x, pp2.y), e3 = fmaf(tf.x, pp2.y, -p3);
                    const float p4 = __fmul_rn(tf.y, pp2.x), e4 = fmaf(tf.y, pp2.x, -p4);
                    const float4 r0 = r0s[k];
                    float sx, ex1, ex2, sy, ey1, ey2;
                    ff rx, ry;
                    two_sum(r0.x, -p1, sx, ex1);
                    two_sum(sx, p2, rx.hi, ex2);
                    rx.lo = __fadd_rn(__fadd_rn(r0.z, __fsub_rn(e2, e1)), __fadd_rn(ex1, ex2));
                    two_sum(r0.y, -p3, sy, ey1);
                    two_sum(sy, -p4, ry.hi, ey2);
                    ry.lo = __fsub_rn(__fadd_rn(r0.w, __fadd_rn(ey1, ey2)), __fadd_rn(e3, e4));
                    if (LARGE) {
                        rx.lo = fmaf(-tf.x, ppl.x, fmaf(tf.y, ppl.y, rx.lo));    // - Re(tau psi_perp,lo)
                        ry.lo = fmaf(-tf.x, ppl.y, fmaf(-tf.y, ppl.x, ry.lo));   // - Im(tau psi_perp,lo)
                    }
                    ff_acc_sq(rr, make_float2(rx.hi, ry.hi));
                    rr.lo = fmaf(2.0f * rx.hi, rx.lo, fmaf(2.0f * ry.hi, ry.lo, rr.lo));
                }
            }
            tc::fence_before_sync();   // TMEM reads complete before the next group's MMAs
        }
        double dlt = J0r - ((double)rr.hi + (double)rr.lo) * ieb64 + dyd;
        if (q > 0.f) {
            const double dx = (double)tf.x - zeta * mr, dyt = (double)tf.y - zeta * mi;
            dlt -= (dx * dx + dyt * dyt) * (double)iq;
            const float alpha_acc = pn * ieb + gg * ieb * ieb;
            dlt -= (double)log1pf(q * alpha_acc);
        }
        delta_sum += dlt;
    }
    if (act) D.lw_y[(size_t)s * P + p] = delta_sum;
    if (bad && (tid & 31) == 0) atomicOr(D.kerr, 1);
    if (tid == 0) {
        // after a timeout: let the copies and MMAs still in flight land (bounded)
        for (int sl = 0; sl < 2; ++sl)
            if ((b_pend >> sl) & 1u) waitB(sl);
        if (n_commit > 0) tc::mbar_wait(mb_mma, (n_commit - 1) & 1u, KAPPA_TC_WAIT);
    }
    tc::fence_before_sync();
    __syncthreads();
    tc::fence_after_sync();
    if (warp == 0) tc::tmem_dealloc(tmem, 256 * NT);
}

// ---------------------------------------------------------------- iota (warp per particle)
// Fast path in FP32: factors from the geometry records, g = Psi^H z, the Gram
// G = Psi^H Psi from the Kronecker factors, Cholesky of eta_bar I + D G D,
// solves, and the element-wise residual (squared sums in FP64).  The FP32
// log det loses accuracy when a pivot cancels, i.e. when a column nearly lies
// in the span of the previous ones (1 - |rho|^2 small, e.g. a fresh birth PF
// next to a real component): each pivot's ratio A_kk / L_kk^2 measures that
// loss, and particles with sqrt(sum ratio^2) > IOTA_RATIO_MAX are queued for
// k_iota_blk, which recomputes them with a float-float Gram and factorisation.
// The FP32 log det error per pivot is about 8 eps ratio (measured), so the
// bound keeps unrepaired particles within ~5e-5 in log-likelihood.
constexpr float IOTA_RATIO_MAX = 100.0f;
constexpr double LOG_PI = 1.14472988584940017414;   // log(pi)

__device__ inline int tri(int i, int j) { return i * (i + 1) / 2 + j; }
__device__ inline void tri_ab(int t, int& a, int& b) {
    a = (int)((sqrtf(8.f * t + 1.f) - 1.f) * 0.5f);
    while ((a + 1) * (a + 2) / 2 <= t) ++a;
    while (a * (a + 1) / 2 > t) --a;
    b = t - a * (a + 1) / 2;
}

// per-warp shared memory of the FP32 path (float2 units)
__host__ __device__ inline size_t iota32_warp_f2(int S, int nfac, int Nf) {
    return (size_t)S * nfac + 4 * (size_t)S + (size_t)S * (S + 1) / 2 + (size_t)S * Nf + (size_t)S;
}

__global__ void k_iota(DevGeom G, DevParams Pm, DevState D, int S, const float* z) {
    extern __shared__ float2 sm32[];
    const int lane = threadIdx.x & 31, wib = threadIdx.x >> 5;
    const int wpb = blockDim.x >> 5;
    const int P = Pm.P, J = G.J, Nz = G.Nz, Nm = G.My * G.Mz, Nf = G.Nf;
    const int nfac = Nf + G.My + G.Mz;
    float2* zs = sm32;                                                    // [Nz]
    float2* base = zs + Nz + wib * iota32_warp_f2(S, nfac, Nf);
    float2* fac = base;                                                   // [S][nfac]
    float2* cS = fac + (size_t)S * nfac;                                  // [S] carrier*amplitude
    float2* cmS = cS + S;                                                 // [S] pi mu, then w
    float2* gS = cmS + S;                                                 // [S] g, rhs, solution
    float2* dS = gS + S;                                                  // [S] (d, A_kk)
    float2* Am = dS + S;                                                  // [S(S+1)/2] packed lower
    float2* gpart = Am + (size_t)S * (S + 1) / 2;                         // [S][Nf] partial g
    const int p = blockIdx.x * wpb + wib;
    const bool act = p < P;
    const int pp = act ? p : 0;
    const float* phi = D.phi[D.cur];
    __shared__ double lg_eb[J_MAX], inv_eb[J_MAX];
    if (threadIdx.x < J) { lg_eb[threadIdx.x] = log(D.eta_bar[threadIdx.x]); inv_eb[threadIdx.x] = 1.0 / D.eta_bar[threadIdx.x]; }
    double total = 0.0;
    float ratio2 = 0.f;
    for (int j = 0; j < J; ++j) {
        __syncthreads();
        for (int k = threadIdx.x; k < Nz; k += blockDim.x)
            zs[k] = make_float2(z[2 * (j * Nz + k)], z[2 * (j * Nz + k) + 1]);
        __syncthreads();
        const double eb = D.eta_bar[j];
        const float ebf = (float)eb;
        // 1. factors and coefficients, lanes over s
        for (int s = lane; s < S; s += 32) {
            const float* ph = phi + (size_t)s * 6 * P;
            float2* fs = fac + (size_t)s * nfac;
            const size_t gi = ((size_t)s * J + j) * P + pp;
            cS[s] = factors_from_geo(G, D.geo[gi], D.geo_lo[gi], fs, fs + Nf, fs + Nf + G.My, 1);
            const float pi = (float)(D.zeta[s * J + j] * D.W[s]);
            const float gm = ph[3 * P + pp], mr = ph[4 * P + pp], mi = ph[5 * P + pp];
            dS[s] = make_float2(sqrtf(fmaxf(pi * (gm + (mr * mr + mi * mi) * (1.0f - pi)), 0.0f)), 0.f);
            cmS[s] = make_float2(pi * mr, pi * mi);
        }
        __syncwarp();
        // 2. g_s = psi_s^H z: tasks (s, f) contract over the antennas, then sum over f
        for (int t = lane; t < S * Nf; t += 32) {
            const int s = t / Nf, f = t - s * Nf;
            const float2* fs = fac + (size_t)s * nfac;
            float2 accy = make_float2(0.f, 0.f);
            for (int y = 0; y < G.My; ++y) {
                float2 accm = make_float2(0.f, 0.f);
                for (int m = 0; m < G.Mz; ++m) {
                    const float2 u = cmulc(fs[Nf + G.My + m], zs[f * Nm + y * G.Mz + m]);
                    accm.x += u.x; accm.y += u.y;
                }
                const float2 u = cmulc(fs[Nf + y], accm);
                accy.x += u.x; accy.y += u.y;
            }
            gpart[t] = cmulc(fs[f], accy);
        }
        // 3. Gram (packed lower) from the Kronecker factors
        const int npair = S * (S + 1) / 2;
        for (int t = lane; t < npair; t += 32) {
            int a, b;
            tri_ab(t, a, b);
            const float2* fa = fac + (size_t)a * nfac;
            const float2* fb2 = fac + (size_t)b * nfac;
            float2 sf = make_float2(0.f, 0.f), sy = sf, sz = sf;
            for (int f = 0; f < Nf; ++f) { const float2 u = cmulc(fa[f], fb2[f]); sf.x += u.x; sf.y += u.y; }
            for (int y = Nf; y < Nf + G.My; ++y) { const float2 u = cmulc(fa[y], fb2[y]); sy.x += u.x; sy.y += u.y; }
            for (int m = Nf + G.My; m < nfac; ++m) { const float2 u = cmulc(fa[m], fb2[m]); sz.x += u.x; sz.y += u.y; }
            Am[t] = cmul(cmulc(cS[a], cS[b]), cmul(sf, cmul(sy, sz)));
        }
        __syncwarp();
        for (int s = lane; s < S; s += 32) {
            float2 acc = make_float2(0.f, 0.f);
            for (int f = 0; f < Nf; ++f) { acc.x += gpart[s * Nf + f].x; acc.y += gpart[s * Nf + f].y; }
            gS[s] = cmulc(cS[s], acc);
        }
        __syncwarp();
        // 4. rhs_a = d_a (g_a - sum_b G_ab cm_b)
        for (int a = lane; a < S; a += 32) {
            float2 acc = gS[a];
            for (int b = 0; b < S; ++b) {
                const float2 gab = (b <= a) ? Am[tri(a, b)] : make_float2(Am[tri(b, a)].x, -Am[tri(b, a)].y);
                const float2 u = cmul(gab, cmS[b]);
                acc.x -= u.x; acc.y -= u.y;
            }
            gS[a] = make_float2(dS[a].x * acc.x, dS[a].x * acc.y);
        }
        __syncwarp();
        // 5. A = eta_bar I + D G D, keep the original diagonal; Cholesky in place
        for (int t = lane; t < npair; t += 32) {
            int a, b;
            tri_ab(t, a, b);
            const float dd = dS[a].x * dS[b].x;
            const float2 v = Am[t];
            Am[t] = make_float2(dd * v.x + (a == b ? ebf : 0.f), dd * v.y);
            if (a == b) dS[a].y = dd * v.x + ebf;
        }
        __syncwarp();
        ffexp det{ff{1.f, 0.f}, 0};
        for (int k = 0; k < S; ++k) {
            const float piv = fmaxf(Am[tri(k, k)].x, 1e-30f);
            const float dk = sqrtf(piv);
            ffexp_mul(det, ff{piv, 0.f});
            const float rk = dS[k].y / piv;
            ratio2 += rk * rk;
            __syncwarp();
            for (int i = k + 1 + lane; i < S; i += 32) {
                const float2 v = Am[tri(i, k)];
                Am[tri(i, k)] = make_float2(v.x / dk, v.y / dk);
            }
            if (lane == 0) Am[tri(k, k)] = make_float2(dk, 0.f);
            __syncwarp();
            const int n = S - k - 1;
            for (int t = lane; t < n * (n + 1) / 2; t += 32) {
                int a, c;
                tri_ab(t, a, c);
                const int i = k + 1 + a, cc = k + 1 + c;
                const float2 u = cmul(Am[tri(i, k)], make_float2(Am[tri(cc, k)].x, -Am[tri(cc, k)].y));
                Am[tri(i, cc)].x -= u.x; Am[tri(i, cc)].y -= u.y;
            }
            __syncwarp();
        }
        // 6. solve L L^H y = rhs
        for (int i = 0; i < S; ++i) {
            float2 acc = make_float2(0.f, 0.f);
            for (int b = lane; b < i; b += 32) { const float2 u = cmul(Am[tri(i, b)], gS[b]); acc.x += u.x; acc.y += u.y; }
            acc.x = warp_sum_f(acc.x); acc.y = warp_sum_f(acc.y);
            if (lane == 0) { const float dd = Am[tri(i, i)].x; gS[i] = make_float2((gS[i].x - acc.x) / dd, (gS[i].y - acc.y) / dd); }
            __syncwarp();
        }
        for (int i = S - 1; i >= 0; --i) {
            float2 acc = make_float2(0.f, 0.f);
            for (int b = i + 1 + lane; b < S; b += 32) { const float2 u = cmulc(Am[tri(b, i)], gS[b]); acc.x += u.x; acc.y += u.y; }
            acc.x = warp_sum_f(acc.x); acc.y = warp_sum_f(acc.y);
            if (lane == 0) { const float dd = Am[tri(i, i)].x; gS[i] = make_float2((gS[i].x - acc.x) / dd, (gS[i].y - acc.y) / dd); }
            __syncwarp();
        }
        // 7. w = cm + d y; |y|^2 (exact squares, float-float sums)
        ff yy{0.f, 0.f};
        for (int a = lane; a < S; a += 32) {
            const float2 y = gS[a];
            ff_acc_sq(yy, y);
            cmS[a] = make_float2(cmS[a].x + dS[a].x * y.x, cmS[a].y + dS[a].x * y.y);
        }
        yy = warp_sum_ff(yy);
        __syncwarp();
        // 8. residual z - sum_s w_s psi_s, element-wise
        ff rr{0.f, 0.f};
        for (int k = lane; k < Nz; k += 32) {
            const int f = k / Nm, ym = k - f * Nm, y = ym / G.Mz, m = ym - y * G.Mz;
            float2 acc = zs[k];
            for (int s = 0; s < S; ++s) {
                const float2* fs = fac + (size_t)s * nfac;
                const float2 u = cmul(cmul(cmS[s], cS[s]), cmul(fs[f], cmul(fs[Nf + y], fs[Nf + G.My + m])));
                acc.x -= u.x; acc.y -= u.y;
            }
            ff_acc_sq(rr, acc);
        }
        rr = warp_sum_ff(rr);
        const double lg = lg_eb[j];
        total += -(ff_to_d(rr) * inv_eb[j] + ff_to_d(yy)) - (ffexp_log(det) - S * lg) - Nz * (LOG_PI + lg);
    }
    if (act && lane == 0) {
        D.lw_x[p] = total;
        if (sqrtf(ratio2) > IOTA_RATIO_MAX) {
            const int slot = atomicAdd(&D.flags[0], 1);
            if (bp_in_range(slot, P, D.kerr)) D.flags[1 + slot] = p;
        }
    }
}

// ---------------------------------------------------------------- iota, float-float Gram and Cholesky
// For the particles the FP32 path flags (or for every particle when S is large):
// the same log-likelihood with the pivots of eta_bar I + D G D kept to ~44 bits,
// so that nearly coinciding columns lose nothing.  One block per
// particle; the lower triangle of A (S <= 64) lives in registers, distributed as
// row pairs (rp, 63 - rp) x column groups c = NCG q + cg (32 NCG threads), so that
// every thread holds about S(S+1)/(64 NCG) entries and every row's scaled column
// entry is formed by NCG threads only.
//  - Gram: G'_ab = (sum_f conj(b'_af) b'_bf)(sum_y ..)(sum_m ..) of the unit-modulus
//    factors, each sum exact to ~2^-40 (products split on a fixed 2^-16 grid,
//    remainders by FMA); A_ab = A_a d_a A_b d_b G'_ab + eta_bar delta_ab in float-float.
//  - Right-looking Cholesky, one barrier per pivot: step k scales column k by
//    1/pivot, subtracts the rank-one term from the trailing entries, and the owners
//    of column k+1 publish it (and its pivot with the reciprocal) for step k+1.
//  - Forward/back solves with the FP32 parts of L, residual in FP32 with FP64 sums
//    (both enter the variational form only at second order).
constexpr int IB_SMAX = 64;
constexpr int IOTA_BLK_NCG = 8;   // column groups: 256 threads, 12 register slots per thread

__device__ inline cff fx_dotc(const float2* x, const float2* y, int n) {
    // sum_k conj(x_k) y_k for |x_k|, |y_k| <= 1 + O(eps), n <= 127: fmaf(a, b, M) - M
    // rounds a*b to a multiple of 2^-16 (M = 1.5 * 2^7), so the grid parts add
    // exactly while |sum| < 256, and fmaf(a, b, -grid part) is the remainder.
    const float M = 192.0f;
    float rh = 0.f, rl = 0.f, ih = 0.f, il = 0.f;
    for (int k = 0; k < n; ++k) {
        const float2 a = x[k], b = y[k];
        float t = __fsub_rn(fmaf(a.x, b.x, M), M);
        rh = __fadd_rn(rh, t); rl = __fadd_rn(rl, fmaf(a.x, b.x, -t));
        t = __fsub_rn(fmaf(a.y, b.y, M), M);
        rh = __fadd_rn(rh, t); rl = __fadd_rn(rl, fmaf(a.y, b.y, -t));
        t = __fsub_rn(fmaf(a.x, b.y, M), M);
        ih = __fadd_rn(ih, t); il = __fadd_rn(il, fmaf(a.x, b.y, -t));
        t = __fsub_rn(fmaf(-a.y, b.x, M), M);
        ih = __fadd_rn(ih, t); il = __fadd_rn(il, fmaf(-a.y, b.x, -t));
    }
    cff r;
    two_sum(rh, rl, r.re.hi, r.re.lo);
    two_sum(ih, il, r.im.hi, r.im.lo);
    return r;
}

// A -= x1 y1 + x2 y2 in float-float: exact high products, first-order cross terms,
// both roundings of the high sum captured; A.lo is left unnormalised.
__device__ inline void ff_sub_dot2(ff& A, ff x1, ff y1, ff x2, ff y2) {
    const float p1 = __fmul_rn(x1.hi, y1.hi), e1 = fmaf(x1.hi, y1.hi, -p1);
    const float p2 = __fmul_rn(x2.hi, y2.hi), e2 = fmaf(x2.hi, y2.hi, -p2);
    float s, t1, t2;
    two_sum(A.hi, -p1, s, t1);
    two_sum(s, -p2, A.hi, t2);
    const float cross = fmaf(x1.hi, y1.lo, fmaf(x1.lo, y1.hi, fmaf(x2.hi, y2.lo, __fmul_rn(x2.lo, y2.hi))));
    A.lo = __fadd_rn(A.lo, __fsub_rn(__fadd_rn(t1, t2), __fadd_rn(__fadd_rn(e1, e2), cross)));
}
// A -= l conj(a)
__device__ inline void cff_sub_mulc(cff& A, const cff& l, const cff& a) {
    ff_sub_dot2(A.re, l.re, a.re, l.im, a.im);
    ff_sub_dot2(A.im, l.im, a.re, ff_neg(l.re), a.im);
}
__device__ inline ff ff_norm(ff x) { ff r; two_sum(x.hi, x.lo, r.hi, r.lo); return r; }
__device__ inline cff cff_norm(cff x) { return cff{ff_norm(x.re), ff_norm(x.im)}; }
__device__ inline ff ff_recip(ff x) {
    const float r = __frcp_rn(x.hi);
    const float e = __fsub_rn(fmaf(-x.hi, r, 1.0f), __fmul_rn(x.lo, r));   // 1 - x r
    ff o;
    fast_two_sum(r, __fmul_rn(r, e), o.hi, o.lo);
    return o;
}

// One trailing entry (i, c) of the factorisation, held as an exact multiple of a
// per-entry grid (h) plus an FP32 remainder (l).  With 2^E >= 4 sqrt(A_ii A_cc),
// every partial Schur complement and every product l_ik conj(l_ck) is below 2^(E-2)
// in modulus (Cauchy-Schwarz for the positive definite A), so fmaf(x, y, M) - M
// (M = 1.5 * 2^E) rounds a product onto the multiples of 2^(E-23), the grid parts
// subtract exactly, and the remainders (exact to 2^(E-48) by FMA) collect in l.
// The row factor enters in float-float, the column factor rounded to FP32: the log
// determinant then stays within ~1e-5 of exact on 64 near-collinear columns.
struct gent { float hr, lr, hi, li, M; };
__device__ inline gent gent_make(const cff& a, float bound) {
    int e;
    frexpf(4.0f * bound, &e);   // 2^e > 4 bound
    gent g;
    g.M = ldexpf(1.5f, e);
    g.hr = __fsub_rn(__fadd_rn(a.re.hi, g.M), g.M);
    g.lr = __fadd_rn(__fsub_rn(a.re.hi, g.hr), a.re.lo);
    g.hi = __fsub_rn(__fadd_rn(a.im.hi, g.M), g.M);
    g.li = __fadd_rn(__fsub_rn(a.im.hi, g.hi), a.im.lo);
    return g;
}
__device__ inline void grid_sub(float& h, float& l, ff x, float y, float M) {   // h + l -= x y
    const float ph = __fsub_rn(fmaf(x.hi, y, M), M);
    h = __fsub_rn(h, ph);
    l = __fsub_rn(l, fmaf(x.lo, y, fmaf(x.hi, y, -ph)));
}
__device__ inline void gent_sub_mulc(gent& g, const cff& x, float2 a) {   // A_ic -= x conj(a)
    grid_sub(g.hr, g.lr, x.re, a.x, g.M);
    grid_sub(g.hr, g.lr, x.im, a.y, g.M);
    grid_sub(g.hi, g.li, x.im, a.x, g.M);
    grid_sub(g.hi, g.li, ff_neg(x.re), a.y, g.M);
}
__device__ inline cff gent_value(const gent& g) {
    cff v;
    two_sum(g.hr, g.lr, v.re.hi, v.re.lo);
    two_sum(g.hi, g.li, v.im.hi, v.im.lo);
    return v;
}

// shared memory of k_iota_blk (bytes): colbuf [2][64] cff, colh [2][64] float2, pivbuf [2][2] ff, red [16]
// double, A packed lower [S(S+1)/2] cff, then float2 z [Nz], factors [S][nfac | 1], cm [S], g [S], L packed [S(S+1)/2]
// (also the partial sums g [S][Nf] before the Gram), then float amplitude [S],
// A d [S], d [S], 1/L_kk [64], pivots [64] ff
__host__ __device__ inline size_t iota_blk_lsize(int S, int Nf) {
    const size_t a = (size_t)S * (S + 1) / 2, b = (size_t)S * Nf;
    return a > b ? a : b;
}
__host__ __device__ inline size_t iota_blk_smem(int S, int nfac, int Nf, int Nz) {
    return 2 * IB_SMAX * 16 + 2 * IB_SMAX * 8 + 4 * 8 + 16 * 8 + (size_t)S * (S + 1) / 2 * 16 +
           ((size_t)Nz + (size_t)S * (nfac | 1) + 2 * (size_t)S + iota_blk_lsize(S, Nf)) * 8 + 3 * (size_t)S * 4 + IB_SMAX * 4 +
           IB_SMAX * 8 +
           // residual: alignment slack, cis table [256] (float4), low parts of the factors [S][nfac | 1]
           16 + 256 * 16 + (size_t)S * (nfac | 1) * 8;
}

// blocks per SM: two 256-thread blocks at 128 registers (67 KB shared each).  Three
// (capped at 80 registers, 112 B spilled) measured 127 ms against 120 ms at 64 x 100k:
// the extra warps against the per-pivot barriers do not pay for the spills
constexpr int IOTA_BLK_PER_SM = 2;

template <int NCG>
__global__ void __launch_bounds__(32 * NCG, IOTA_BLK_PER_SM) k_iota_blk(DevGeom G, DevParams Pm, DevState D, int S, const float* z, int all) {
    constexpr int IB_T = 32 * NCG;
    constexpr int QA = 32 / NCG, QB = 64 / NCG;   // register slots of rows ra (< 32) and rb (>= 32)
    extern __shared__ float4 smb[];
    cff* colbuf = reinterpret_cast<cff*>(smb);                    // [2][IB_SMAX] published column (row side)
    float2* colh = reinterpret_cast<float2*>(colbuf + 2 * IB_SMAX);   // [2][IB_SMAX] same, rounded (column side)
    ff* pivbuf = reinterpret_cast<ff*>(colh + 2 * IB_SMAX);       // [2][piv, 1/piv]
    double* red = reinterpret_cast<double*>(pivbuf + 4);          // [16]: yy, then per-warp |r|^2 at 8 + warp
    const int P = Pm.P, J = G.J, Nz = G.Nz, Nm = G.My * G.Mz, Nf = G.Nf;
    const int nfac = (Nf + G.My + G.Mz) | 1;   // factor row stride, odd in float2 against bank conflicts
    cff* Apk = reinterpret_cast<cff*>(red + 16);                   // [S(S+1)/2] float-float A
    float2* zs = reinterpret_cast<float2*>(Apk + (size_t)S * (S + 1) / 2);   // [Nz]
    float2* fac = zs + Nz;                                        // [S][nfac]: b', a_y, a_z
    float2* cmS = fac + (size_t)S * nfac;                         // [S] pi mu, then A (pi mu + d y)
    float2* gS = cmS + S;                                         // [S] g, rhs, solution
    float2* Lsm = gS + S;                                         // FP32 G, then L (packed lower)
    float2* gpart = Lsm;                                          // [S][Nf] (before the Gram)
    float* amp = reinterpret_cast<float*>(Lsm + iota_blk_lsize(S, Nf));     // [S]
    float* adS = amp + S;                                         // [S] A d
    float* dS = adS + S;                                          // [S] d
    float* ild = dS + S;                                          // [IB_SMAX] 1 / L_kk
    ff* pivs = reinterpret_cast<ff*>(ild + IB_SMAX);              // [IB_SMAX] pivots
    // [256] e^{i 2 pi n / 256} (hi, lo), on a 16-byte boundary (the float arrays above end on 4)
    float4* ctab = reinterpret_cast<float4*>((reinterpret_cast<uintptr_t>(pivs + IB_SMAX) + 15) & ~(uintptr_t)15);
    float2* flo = reinterpret_cast<float2*>(ctab + 256);          // [S][nfac] low parts of the factors
    const int tid = threadIdx.x, lane = tid & 31, wid = tid >> 5;
    const int cg = lane % NCG;
    const int rp = wid * (32 / NCG) + lane / NCG;
    const int ra = rp, rb = IB_SMAX - 1 - rp;
    const float* phi = D.phi[D.cur];
    __shared__ double lg_eb[J_MAX], inv_eb[J_MAX];
    if (tid < J) { lg_eb[tid] = log(D.eta_bar[tid]); inv_eb[tid] = 1.0 / D.eta_bar[tid]; }
    cis_table_fill(ctab, tid, IB_T);
    const int count = all ? P : D.flags[0];
    for (int w = blockIdx.x; w < count; w += gridDim.x) {
        const int pp = all ? w : D.flags[1 + w];
        double total = 0.0;
        for (int j = 0; j < J; ++j) {
            __syncthreads();
            for (int k = tid; k < Nz; k += IB_T) zs[k] = make_float2(z[2 * (j * Nz + k)], z[2 * (j * Nz + k) + 1]);
            const double eb = D.eta_bar[j];
            const float ebf = (float)eb;
            const ff ebff = ff{ebf, (float)(eb - (double)ebf)};
            for (int s = tid; s < S; s += IB_T) {
                const float* ph = phi + (size_t)s * 6 * P;
                float2* fs = fac + (size_t)s * nfac;
                const size_t gi = ((size_t)s * J + j) * P + pp;
                const float A = factors_from_geo_pairs(G, ctab, D.geo[gi], D.geo_lo[gi], fs, flo + (size_t)s * nfac);
                const float pi = (float)(D.zeta[s * J + j] * D.W[s]);
                const float gm = ph[3 * P + pp], mr = ph[4 * P + pp], mi = ph[5 * P + pp];
                const float d = sqrtf(fmaxf(pi * (gm + (mr * mr + mi * mi) * (1.0f - pi)), 0.0f));
                amp[s] = A;
                dS[s] = d;
                adS[s] = A * d;
                cmS[s] = make_float2(pi * mr, pi * mi);
            }
            __syncthreads();
            // g_s = psi_s^H z: tasks (s, f) contract over the antennas
            for (int t = tid; t < S * Nf; t += IB_T) {
                const int f = t / S, s = t - f * S;   // lanes over s: z_f broadcast
                const float2* fs = fac + (size_t)s * nfac;
                float2 accy = make_float2(0.f, 0.f);
                for (int y = 0; y < G.My; ++y) {
                    float2 accm = make_float2(0.f, 0.f);
                    for (int m = 0; m < G.Mz; ++m) {
                        const float2 u = cmulc(fs[Nf + G.My + m], zs[f * Nm + y * G.Mz + m]);
                        accm.x += u.x; accm.y += u.y;
                    }
                    const float2 u = cmulc(fs[Nf + y], accm);
                    accy.x += u.x; accy.y += u.y;
                }
                gpart[s * Nf + f] = cmulc(fs[f], accy);
            }
            __syncthreads();
            for (int s = tid; s < S; s += IB_T) {
                float2 acc = make_float2(0.f, 0.f);
                for (int f = 0; f < Nf; ++f) { acc.x += gpart[s * Nf + f].x; acc.y += gpart[s * Nf + f].y; }
                gS[s] = make_float2(amp[s] * acc.x, amp[s] * acc.y);
            }
            __syncthreads();
            // Gram, one packed entry per task (a >= b), into shared memory
            for (int t = tid; t < S * (S + 1) / 2; t += IB_T) {
                int a, b;
                tri_ab(t, a, b);
                const float2* fa = fac + (size_t)a * nfac;
                const float2* fb = fac + (size_t)b * nfac;
                const cff sf = fx_dotc(fa, fb, Nf);
                const cff sy = fx_dotc(fa + Nf, fb + Nf, G.My);
                const cff sz = fx_dotc(fa + Nf + G.My, fb + Nf + G.My, G.Mz);
                const cff gu = cff_mul(sf, cff_mul(sy, sz));
                const float aa = amp[a] * amp[b];
                Lsm[t] = make_float2(aa * (gu.re.hi + gu.re.lo), aa * (gu.im.hi + gu.im.lo));
                const ff sc = ff_prod(adS[a], adS[b]);
                cff v{ff_mul(gu.re, sc), ff_mul(gu.im, sc)};
                if (a == b) { v.re = ff_add(v.re, ebff); v.im = ff{0.f, 0.f}; }
                Apk[t] = v;
                if (b == 0) { colbuf[a] = v; colh[a] = make_float2(v.re.hi, v.im.hi); }
                if (t == 0) { pivbuf[0] = v.re; pivbuf[1] = ff_recip(v.re); }
            }
            __syncthreads();
            // this thread's slots (rows ra: q < 8, rb: q < 16) into registers
            gent Ar[QA], Br[QB];
            unsigned liveA = 0u, liveB = 0u;   // slots of the lower triangle; cleared as columns finish
            {
                const float sa = (ra < S) ? sqrtf(Apk[tri(ra, ra)].re.hi) : 0.f;
                const float sb = (rb < S) ? sqrtf(Apk[tri(rb, rb)].re.hi) : 0.f;
                #pragma unroll
                for (int q = 0; q < QA; ++q) {
                    const int c = NCG * q + cg;
                    if (c <= ra && ra < S) { Ar[q] = gent_make(Apk[tri(ra, c)], sa * sqrtf(Apk[tri(c, c)].re.hi)); liveA |= 1u << q; }
                }
                #pragma unroll
                for (int q = 0; q < QB; ++q) {
                    const int c = NCG * q + cg;
                    if (c <= rb && rb < S) { Br[q] = gent_make(Apk[tri(rb, c)], sb * sqrtf(Apk[tri(c, c)].re.hi)); liveB |= 1u << q; }
                }
            }
            // rhs_a = d_a (g_a - sum_b G_ab pi_b mu_b), FP32
            float2 rhs = make_float2(0.f, 0.f);
            const int fst = tid - 64;   // forward-substitution row of this thread (warps 2-3)
            if (fst >= 0 && fst < S) {
                const int a = fst;
                float2 acc = gS[a];
                for (int b = 0; b < S; ++b) {
                    const float2 e = (b <= a) ? Lsm[tri(a, b)] : make_float2(Lsm[tri(b, a)].x, -Lsm[tri(b, a)].y);
                    const float2 u = cmul(e, cmS[b]);
                    acc.x -= u.x; acc.y -= u.y;
                }
                rhs = make_float2(dS[a] * acc.x, dS[a] * acc.y);
            }
            __syncthreads();
            // Cholesky with exactly accumulated trailing entries; log det from the
            // float-float product of the pivots (exponent kept apart)
            for (int k = 0; k < S; ++k) {
                const int cur = k & 1, nxt = cur ^ 1;
                const cff* col = colbuf + cur * IB_SMAX;
                const float2* colr = colh + cur * IB_SMAX;
                cff* ncol = colbuf + nxt * IB_SMAX;
                float2* ncolr = colh + nxt * IB_SMAX;
                ff piv = pivbuf[2 * cur];
                ff inv = pivbuf[2 * cur + 1];
                if (!(piv.hi > 0.f)) { piv = ff{1e-30f, 0.f}; inv = ff{1e30f, 0.f}; }
                // FP32 factor for the (variational) solves: 1/L_kk by the fast reciprocal square root
                const float il = rsqrtf(piv.hi + piv.lo);
                const float lkk = (piv.hi + piv.lo) * il;
                // column c = NCG q + cg takes updates while c > k: the slot of column k retires
                const int kc = k - cg;
                if (kc >= 0 && kc % NCG == 0) { liveA &= ~(1u << (kc / NCG)); liveB &= ~(1u << (kc / NCG)); }
                if (tid == 0) {
                    pivs[k] = piv;
                    Lsm[tri(k, k)] = make_float2(lkk, 0.f);
                    ild[k] = il;
                }
                // forward substitution L u = rhs, one column behind the factorisation:
                // row i takes column k-1 (published last step), then row k yields u_k
                if (fst >= k && fst < S) {
                    if (k > 0) {
                        const float2 u = cmul(Lsm[tri(fst, k - 1)], gS[k - 1]);
                        rhs.x -= u.x; rhs.y -= u.y;
                    }
                    if (fst == k) gS[k] = make_float2(rhs.x * il, rhs.y * il);
                }
                {   // FP32 column k of L for the solves (warps 4-5)
                    const int i = k + 1 + (tid - 128);
                    if (tid >= 128 && i < S) {
                        const cff v = col[i];
                        Lsm[tri(i, k)] = make_float2((v.re.hi + v.re.lo) * il, (v.im.hi + v.im.lo) * il);
                    }
                }
                cff la{}, lb{};
                if (ra > k && ra < S) { const cff v = col[ra]; la = cff{ff_mul(v.re, inv), ff_mul(v.im, inv)}; }
                if (rb > k && rb < S) { const cff v = col[rb]; lb = cff{ff_mul(v.re, inv), ff_mul(v.im, inv)}; }
                #pragma unroll
                for (int q = 0; q < QA; ++q) {
                    const int c = NCG * q + cg;
                    if (liveA & (1u << q)) {
                        gent_sub_mulc(Ar[q], la, colr[c]);
                        if (NCG * q == kc + 1) {
                            const cff v = gent_value(Ar[q]);
                            ncol[ra] = v;
                            ncolr[ra] = make_float2(v.re.hi, v.im.hi);
                            if (ra == c) { pivbuf[2 * nxt] = v.re; pivbuf[2 * nxt + 1] = ff_recip(v.re); }
                        }
                    }
                }
                #pragma unroll
                for (int q = 0; q < QB; ++q) {
                    const int c = NCG * q + cg;
                    if (liveB & (1u << q)) {
                        gent_sub_mulc(Br[q], lb, colr[c]);
                        if (NCG * q == kc + 1) {
                            const cff v = gent_value(Br[q]);
                            ncol[rb] = v;
                            ncolr[rb] = make_float2(v.re.hi, v.im.hi);
                            if (rb == c) { pivbuf[2 * nxt] = v.re; pivbuf[2 * nxt + 1] = ff_recip(v.re); }
                        }
                    }
                }
                __syncthreads();
            }
            // back substitution L^H y = u (warp 0; lane owns rows lane and lane + 32); log det
            // from the float-float product of the pivots (exponents apart)
            if (wid == 0) {
                ffexp det{ff{1.f, 0.f}, 0};
                for (int k = lane; k < S; k += 32) ffexp_mul(det, pivs[k]);
                #pragma unroll
                for (int o = 16; o > 0; o >>= 1) {
                    const ff om{__shfl_xor_sync(0xffffffffu, det.m.hi, o), __shfl_xor_sync(0xffffffffu, det.m.lo, o)};
                    const int oe = __shfl_xor_sync(0xffffffffu, det.e, o);
                    ffexp_mul(det, om);
                    det.e += oe;
                }
                if (lane == 0) red[1] = ffexp_log(det);
                float2 r0 = (lane < S) ? gS[lane] : make_float2(0.f, 0.f);
                float2 r1 = (lane + 32 < S) ? gS[lane + 32] : make_float2(0.f, 0.f);
                const float i0 = (lane < S) ? ild[lane] : 0.f, i1 = (lane + 32 < S) ? ild[lane + 32] : 0.f;
                for (int k = S - 1; k >= 0; --k) {
                    const float2 lr0 = (lane < k) ? Lsm[tri(k, lane)] : make_float2(0.f, 0.f);
                    const float2 lr1 = (lane + 32 < k) ? Lsm[tri(k, lane + 32)] : make_float2(0.f, 0.f);
                    const bool hi_row = k >= 32;
                    const float2 own = hi_row ? r1 : r0;
                    const float io = hi_row ? i1 : i0;
                    const float2 yk = make_float2(__shfl_sync(0xffffffffu, own.x * io, k & 31),
                                                  __shfl_sync(0xffffffffu, own.y * io, k & 31));
                    if (lane == (k & 31)) { if (hi_row) r1 = yk; else r0 = yk; }
                    if (lane < k) { const float2 u = cmulc(lr0, yk); r0.x -= u.x; r0.y -= u.y; }
                    if (lane + 32 < k) { const float2 u = cmulc(lr1, yk); r1.x -= u.x; r1.y -= u.y; }
                }
                ff yy{0.f, 0.f};
                if (lane < S) {
                    ff_acc_sq(yy, r0);
                    const float2 c = cmS[lane];
                    cmS[lane] = make_float2(amp[lane] * (c.x + dS[lane] * r0.x), amp[lane] * (c.y + dS[lane] * r0.y));
                }
                if (lane + 32 < S) {
                    ff_acc_sq(yy, r1);
                    const float2 c = cmS[lane + 32];
                    cmS[lane + 32] = make_float2(amp[lane + 32] * (c.x + dS[lane + 32] * r1.x),
                                                 amp[lane + 32] * (c.y + dS[lane + 32] * r1.y));
                }
                yy = warp_sum_ff(yy);
                if (lane == 0) red[0] = ff_to_d(yy);
            }
            __syncthreads();
            // residual r = z - sum_s w_s (b' kron a_y kron a_z)_s, w_s = A_s (pi mu + d y)_s.  Its
            // energy reaches ~1e4 noise units, so the steering values enter as (hi, lo) pairs
            // (~1e-9), the products of the high parts are summed exactly on a grid fixed for
            // this (p, j) (2^E > 4 (max_k |z_k| + sum_s |w_s|) bounds every partial sum), and
            // the remainders and the low-part cross terms are summed in FP32
            if (wid == 1) {
                float b = 0.f, zm = 0.f;
                for (int s = lane; s < S; s += 32) b += fabsf(cmS[s].x) + fabsf(cmS[s].y);
                for (int k = lane; k < Nz; k += 32) zm = fmaxf(zm, fabsf(zs[k].x) + fabsf(zs[k].y));
                b = warp_sum_f(b);
                #pragma unroll
                for (int o = 16; o > 0; o >>= 1) zm = fmaxf(zm, __shfl_xor_sync(0xffffffffu, zm, o));
                if (lane == 0) red[2] = (double)(b + zm);
            }
            __syncthreads();
            int gE;
            frexpf(4.0f * (float)red[2] + 1e-30f, &gE);
            const float GM = ldexpf(1.5f, gE);
            ff rr{0.f, 0.f};
            for (int k = tid; k < Nz; k += IB_T) {
                const int f = k / Nm, ym = k - f * Nm, y = ym / G.Mz, m = ym - y * G.Mz;
                const float2 zk = zs[k];
                float2 gr, rm;
                gr.x = __fsub_rn(__fadd_rn(zk.x, GM), GM);
                gr.y = __fsub_rn(__fadd_rn(zk.y, GM), GM);
                rm.x = __fsub_rn(zk.x, gr.x);
                rm.y = __fsub_rn(zk.y, gr.y);
                for (int s = 0; s < S; ++s) {
                    // w_s (FP32, exact) times psi'_sk = b'_f a_y a_z as a (hi, lo) pair
                    const float2* fs = fac + (size_t)s * nfac;
                    const float2* fl = flo + (size_t)s * nfac;
                    const float4 ay = cpair_mul(fs[Nf + y], fl[Nf + y], fs[Nf + G.My + m], fl[Nf + G.My + m]);
                    const float4 c = cpair_mul(fs[f], fl[f], make_float2(ay.x, ay.y), make_float2(ay.z, ay.w));
                    const float2 u = cmS[s];
                    float t;
                    t = __fsub_rn(fmaf(u.x, c.x, GM), GM); gr.x = __fsub_rn(gr.x, t); rm.x -= fmaf(u.x, c.x, -t);
                    t = __fsub_rn(fmaf(-u.y, c.y, GM), GM); gr.x = __fsub_rn(gr.x, t); rm.x -= fmaf(-u.y, c.y, -t);
                    t = __fsub_rn(fmaf(u.x, c.y, GM), GM); gr.y = __fsub_rn(gr.y, t); rm.y -= fmaf(u.x, c.y, -t);
                    t = __fsub_rn(fmaf(u.y, c.x, GM), GM); gr.y = __fsub_rn(gr.y, t); rm.y -= fmaf(u.y, c.x, -t);
                    rm.x -= fmaf(u.x, c.z, -u.y * c.w);
                    rm.y -= fmaf(u.x, c.w, u.y * c.z);
                }
                float hx, lx, hy, ly;
                two_sum(gr.x, rm.x, hx, lx);
                two_sum(gr.y, rm.y, hy, ly);
                ff_acc_sq(rr, make_float2(hx, hy));
                rr.lo = fmaf(2.0f * hx, lx, fmaf(2.0f * hy, ly, rr.lo));
            }
            rr = warp_sum_ff(rr);
            if (lane == 0) red[8 + wid] = ff_to_d(rr);
            __syncthreads();
            if (tid == 0) {
                double rrs = 0.0;
                for (int w2 = 0; w2 < IB_T / 32; ++w2) rrs += red[8 + w2];
                const double lg = lg_eb[j];
                total += -(rrs * inv_eb[j] + red[0]) - (red[1] - S * lg) - Nz * (LOG_PI + lg);
            }
        }
        if (tid == 0) D.lw_x[pp] = total;
    }
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

// B tiles of the tensor-core pass 1, once per (s, j, round r of elements 16 r .. 16 r + 15):
// rows n of [[Re V, Im V], [Im V, -Re V]]^T (n < SW: Re h_n, n >= SW: Im h_{n-SW}, SW = SCA
// basis columns incl. r0) against the real K index 2 e + part of the round's element e
// (part 0 = Re psi, 1 = Im psi; zero past the last element), split into TF32 high and low
// parts, in the K-major core-matrix layout; [hi, lo] per round.
__global__ void k_kappa_btile(DevGeom G, DevState D, int SCA, float* __restrict__ Bt) {
    constexpr int KR = KAPPA_TC_KR;
    const int s = blockIdx.x, j = blockIdx.y, r = blockIdx.z;
    const int J = G.J, Nz = G.Nz, Nm = G.My * G.Mz, N1 = 2 * SCA;
    const int R1 = kappa_tc_r1(G.Nf, Nm);
    const float2* V = D.kV + ((size_t)s * J + j) * Nz * SCA;
    float* out = Bt + (((size_t)s * J + j) * R1 + r) * 2 * N1 * KR;
    for (int t = threadIdx.x; t < N1 * KR; t += blockDim.x) {
        const int n = t / KR, kk = t - n * KR;
        const int k = r * 16 + (kk >> 1), part = kk & 1;
        const int c = n < SCA ? n : n - SCA;
        const float2 v = (k < Nz) ? V[(size_t)k * SCA + c] : make_float2(0.f, 0.f);
        const float b = (n < SCA) ? (part == 0 ? v.x : v.y) : (part == 0 ? v.y : -v.x);
        const float hi = tc::tf32_rn(b);
        const int off = tc::core_off(n, kk, KR) >> 2;
        out[off] = hi;
        out[N1 * KR + off] = tc::tf32_rn(b - hi);
    }
}

// B tiles of the tensor-core pass 2, once per (s, j, group g of elements 32 g .. 32 g + 31,
// K chunk kc of SCA / 16): rows n < nkp are the real parts, rows nkp <= n < 2 nkp the
// imaginary parts of the group's elements e (rows past the group's nk elements are zero),
// against the real K index 2 (c - 16 kc) + part of basis columns c (part 0 = Re h_c,
// 1 = Im h_c; the r0 column SCA - 1 excluded): Re row [Re V_ec, Im V_ec], Im row
// [Im V_ec, -Re V_ec]; TF32 hi/lo, K-major core-matrix layout, [hi, lo] per slot of
// 2 x 64 x 32 floats.
__global__ void k_kappa_btile2(DevGeom G, DevState D, int SCA, float* __restrict__ Bt2) {
    constexpr int KC2 = KAPPA_TC_KC2;
    const int NCH = SCA / 16;
    const int s = blockIdx.x, j = blockIdx.y, g = blockIdx.z / NCH, kc = blockIdx.z - g * NCH;
    const int J = G.J, Nz = G.Nz, Nm = G.My * G.Mz, NG = kappa_tc_groups(G.Nf, Nm);
    const int k0 = 32 * g, nk = min(32, Nz - k0), nkp = round16(nk), N2 = 2 * nkp;
    const float2* V = D.kV + ((size_t)s * J + j) * Nz * SCA;
    float* out = Bt2 + ((((size_t)s * J + j) * NG + g) * NCH + kc) * (size_t)(2 * KAPPA_TC_N2 * KC2);
    for (int t = threadIdx.x; t < N2 * KC2; t += blockDim.x) {
        const int n = t / KC2, kk = t - n * KC2;
        const bool im = n >= nkp;
        const int e = im ? n - nkp : n;
        const int c = kc * 16 + (kk >> 1), part = kk & 1;
        float2 v = make_float2(0.f, 0.f);
        if (e < nk && c < SCA - 1) v = V[(size_t)(k0 + e) * SCA + c];
        const float b = im ? (part == 0 ? v.y : -v.x) : (part == 0 ? v.x : v.y);
        const float hi = tc::tf32_rn(b);
        const int off = tc::core_off(n, kk, KC2) >> 2;
        out[off] = hi;
        out[N2 * KC2 + off] = tc::tf32_rn(b - hi);
    }
}

// dynamic shared memory of k_kappa_tc: the operand region (pass 1: A [NT][hi, lo][128 x 32],
// B [hi, lo][2 SW x 32]; pass 2: A [NT][hi, lo][128 x 32], two B slots [hi, lo][64 x 32]),
// barriers, r0 (hi, lo) per element, 1/lambda_c and y~0_c, and the factors of 128 NT particles
constexpr int KAPPA_TC_NT = 1;   // M tiles per block of the launched variant
static bool kappa_tc_large(const DevGeom& G) {
    const int Nm = G.My * G.Mz;
    return Nm >= 32 && Nm % 16 == 0;
}
static size_t kappa_tc_smem(const DevGeom& G, int SW, int NT = KAPPA_TC_NT) {
    const bool large = kappa_tc_large(G);
    const size_t nfac = (size_t)(large || G.Nf > KAPPA_TC_FLY_NF ? 0 : G.Nf) + G.My + G.Mz;
    const size_t rf = (size_t)kappa_tc_region_floats(SW, NT);
    const size_t pairs = large ? (size_t)G.Mz * 128 * NT * sizeof(float2) + 16 + 256 * sizeof(float4) : 0;
    return rf * sizeof(float) + 32 + (size_t)G.Nz * sizeof(float4) + 2 * (size_t)SW * sizeof(float2) +
           nfac * 128 * NT * sizeof(float2) + pairs;
}
// The tensor-core variant applies to
//   * 64 basis columns (SCA = 64) with 2 My Mz in {8, 16, 32} (a pass-1 round is whole
//     frequencies), and
//   * 64 or 32 basis columns with My Mz a multiple of 16, at least 32 (a round is part of
//     one frequency; the large arrays, whose CUDA-core kernel stages few frequencies),
// both with Mz even (a pass-1 round writes the pairs (m, m + 1) of a row) and the shared
// memory within the opt-in limit.  The tensor core adds each MMA's result into its FP32
// accumulator (no FMA chain): with 75 frequencies of the 2 x 2 URA in one pass-1
// accumulator (225 accumulations) the PF weights moved by 1.7e-4 (measured), with 24 they
// stayed within 1e-4; hence the segments of KAPPA_TC_SEG rounds.
bool kappa_tc_ok(const DevGeom& G, int SCA) {
    const int Nm = G.My * G.Mz, KC = 2 * Nm;
    if (G.Mz % 2 != 0) return false;
    const bool whole = SCA == 64 && (KC == 8 || KC == 16 || KC == 32);
    const bool part = (SCA == 64 || SCA == 32) && kappa_tc_large(G);
    return (whole || part) && kappa_tc_smem(G, SCA) <= 227 * 1024;
}
static size_t kappa_btile1_floats(const DevGeom& G, int S_max, int SCA) {
    return (size_t)S_max * G.J * kappa_tc_r1(G.Nf, G.My * G.Mz) * 2 * (2 * SCA) * KAPPA_TC_KR;
}
size_t kappa_btile_floats(const DevGeom& G, int S_max, int SCA) {
    const int Nm = G.My * G.Mz;
    return kappa_btile1_floats(G, S_max, SCA) +
           (size_t)S_max * G.J * kappa_tc_groups(G.Nf, Nm) * (SCA / 16) * (2 * KAPPA_TC_N2 * KAPPA_TC_KC2);
}
int launch_kappa_btile(const DevGeom& G, const DevState& D, int S, int SCA, cudaStream_t st) {
    if (!D.kB || !kappa_tc_ok(G, SCA)) return 0;
    const int Nm = G.My * G.Mz;
    k_kappa_btile<<<dim3(S, G.J, kappa_tc_r1(G.Nf, Nm)), 256, 0, st>>>(G, D, SCA, D.kB);
    k_kappa_btile2<<<dim3(S, G.J, kappa_tc_groups(G.Nf, Nm) * (SCA / 16)), 256, 0, st>>>(
        G, D, SCA, D.kB + kappa_btile1_floats(G, S, SCA));
    return 2;
}

// shared memory of the CUDA-core PF likelihood: 1/lambda, y~0 [2 SC], factors [nfac][256],
// low parts of a_y, a_z [My + Mz][256] (float2), alignment slack and the (hi, lo) cis table
// [256] (float4), then per staged frequency the V rows, the low part of r0 and |V_k|^2
static size_t kappa_smem_fixed(const DevGeom& G, int SC) {
    const size_t nfac = (size_t)G.Nf + G.My + G.Mz;
    return (2 * (size_t)SC + (nfac + G.My + G.Mz) * 256) * sizeof(float2) + 16 + 256 * sizeof(float4);
}
static size_t kappa_smem_per_f(const DevGeom& G, int SC) {
    const size_t Nm = (size_t)G.My * G.Mz;
    return Nm * (SC + 1) * sizeof(float2) + Nm * sizeof(float);
}
// shared-memory budget per block: one block per SM, or two (228 KB per SM, 1 KB reserved each)
static size_t kappa_smem_budget(int mb) { return mb == 2 ? 112 * 1024 : 200 * 1024; }

static bool kappa_sc_valid(int sc) { return sc == 8 || sc == 16 || sc == 24 || sc == 32 || sc == 48 || sc == 64; }

KappaPlan plan_kappa(const DevGeom& G, const DevState& D, int S, int SCA, int t_sc, int t_mb, int t_fch, int t_tc) {
    KappaPlan k{};
    // the bucket: the requested one where it holds S and fits the basis stride, else the
    // smallest that holds S; the tensor-core kernel where allowed and not declined
    // (the kernel's width is the basis stride: 64, or 32 for the large arrays)
    const bool tc_shape = D.kB && kappa_tc_ok(G, SCA);
    if (kappa_sc_valid(t_sc) && t_sc >= S && t_sc <= SCA) k.sc = t_sc;
    else if (S > 32 && tc_shape && t_tc >= 0) k.sc = 64;
    else k.sc = S <= 8 ? 8 : S <= 16 ? 16 : S <= 24 ? 24 : S <= 32 ? 32 : S <= 48 ? 48 : 64;
    k.tc = k.sc == SCA && tc_shape && t_tc >= 0;
    if (k.tc) return k;
    k.mb = (k.sc <= 16) ? 2 : (t_mb == 2 && k.sc <= 32 ? 2 : 1);
    const size_t fixed = kappa_smem_fixed(G, k.sc), per_f = kappa_smem_per_f(G, k.sc);
    if (k.mb == 2 && k.sc > 16 && fixed + per_f > kappa_smem_budget(2)) k.mb = 1;
    const size_t limit = kappa_smem_budget(k.mb);
    int fch = G.Nf;
    while (fch > 1 && fixed + fch * per_f > limit) fch = (fch + 1) / 2;
    if (t_fch > 0 && t_fch < fch) fch = t_fch;
    k.fch = fch;
    k.smem = fixed + (size_t)fch * per_f;
    return k;
}

template <int SC, int MB>
static void launch_kappa_cc(const DevGeom& G, const DevParams& Pm, const DevState& D, int S, int SCA, int fch,
                            size_t smem, cudaStream_t st) {
    smem_allow_max((const void*)k_kappa<SC, MB>);
    k_kappa<SC, MB><<<dim3((Pm.P + 255) / 256, S), 256, smem, st>>>(G, Pm, D, S, SCA, fch);
}

void launch_kappa(const DevGeom& G, const DevParams& Pm, const DevState& D, int S, int SCA, const KappaPlan& k,
                  cudaStream_t st) {
    if (k.tc) {
        constexpr int NT = KAPPA_TC_NT;
        const dim3 grid((Pm.P + 128 * NT - 1) / (128 * NT), S);
        const float* bt2 = D.kB + kappa_btile1_floats(G, S, SCA);
        if (!kappa_tc_large(G)) {
            smem_allow_max((const void*)k_kappa_tc<NT, 64, false>);
            k_kappa_tc<NT, 64, false><<<grid, 128 * NT, kappa_tc_smem(G, 64), st>>>(G, Pm, D, S, SCA, D.kB, bt2);
        } else if (SCA == 64) {
            smem_allow_max((const void*)k_kappa_tc<NT, 64, true>);
            k_kappa_tc<NT, 64, true><<<grid, 128 * NT, kappa_tc_smem(G, 64), st>>>(G, Pm, D, S, SCA, D.kB, bt2);
        } else {
            smem_allow_max((const void*)k_kappa_tc<NT, 32, true>);
            k_kappa_tc<NT, 32, true><<<grid, 128 * NT, kappa_tc_smem(G, 32), st>>>(G, Pm, D, S, SCA, D.kB, bt2);
        }
        return;
    }
    switch (k.sc * 4 + k.mb) {
        case 8 * 4 + 2:  launch_kappa_cc<8, 2>(G, Pm, D, S, SCA, k.fch, k.smem, st); break;
        case 16 * 4 + 2: launch_kappa_cc<16, 2>(G, Pm, D, S, SCA, k.fch, k.smem, st); break;
        case 24 * 4 + 1: launch_kappa_cc<24, 1>(G, Pm, D, S, SCA, k.fch, k.smem, st); break;
        case 24 * 4 + 2: launch_kappa_cc<24, 2>(G, Pm, D, S, SCA, k.fch, k.smem, st); break;
        case 32 * 4 + 1: launch_kappa_cc<32, 1>(G, Pm, D, S, SCA, k.fch, k.smem, st); break;
        case 32 * 4 + 2: launch_kappa_cc<32, 2>(G, Pm, D, S, SCA, k.fch, k.smem, st); break;
        case 48 * 4 + 1: launch_kappa_cc<48, 1>(G, Pm, D, S, SCA, k.fch, k.smem, st); break;
        default:         launch_kappa_cc<64, 1>(G, Pm, D, S, SCA, k.fch, k.smem, st); break;
    }
}

// S below which the FP32 path runs first and only flagged particles are redone
constexpr int IOTA_FF_ALL_S = 24;

int launch_iota(const DevGeom& G, const DevParams& Pm, const DevState& D, int S, const float* z, cudaStream_t st) {
    if (S >= IOTA_FF_ALL_S) return launch_iota_bulk(G, Pm, D, S, z, st);
    const int nfac = G.Nf + G.My + G.Mz;
    const size_t per_warp = iota32_warp_f2(S, nfac, G.Nf) * sizeof(float2);
    int wpb = 8;
    while (wpb > 1 && (size_t)G.Nz * sizeof(float2) + wpb * per_warp > 64 * 1024) wpb /= 2;
    const size_t smem = (size_t)G.Nz * sizeof(float2) + wpb * per_warp;
    cudaMemsetAsync(D.flags, 0, sizeof(int), st);
    smem_allow_max((const void*)k_iota);
    k_iota<<<(Pm.P + wpb - 1) / wpb, 32 * wpb, smem, st>>>(G, Pm, D, S, z);
    return 1;
}

void launch_iota_repair(const DevGeom& G, const DevParams& Pm, const DevState& D, int S, const float* z, cudaStream_t st) {
    const int nfac = G.Nf + G.My + G.Mz;
    const size_t smem = iota_blk_smem(S, nfac, G.Nf, G.Nz);
    constexpr int NCG = IOTA_BLK_NCG;
    smem_allow_max((const void*)k_iota_blk<NCG>);
    int sms = 0, dev = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    const int wave = IOTA_BLK_PER_SM * std::max(sms, 1);
    k_iota_blk<NCG><<<wave, 32 * NCG, smem, st>>>(G, Pm, D, S, z, 0);
}

void launch_nu(const DevGeom& G, const DevParams& Pm, const DevState& D, int S, cudaStream_t st) {
    const int n = G.J * Pm.P;
    k_nu<<<(n + 255) / 256, 256, 0, st>>>(G, Pm, D, S);
}

}  // namespace bp

namespace bp {
size_t iota_blk_smem_bytes(const DevGeom& G, int S) {
    return iota_blk_smem(S, G.Nf + G.My + G.Mz, G.Nf, G.Nz);
}
}  // namespace bp
