// MT likelihood iota~ (Supplementary Sec. S-V) of every particle in FP32, with an
// error bound per particle, and the selection of the particles whose weights need
// the float-float evaluation of k_iota_blk.
//
// Per (p, j) the message is log iota~ = -Nz log pi - log det C - e^H C^-1 e with
// C = eta_bar I + Psi D^2 Psi^H and e = z - Psi (pi mu).  With A = eta_bar I + D G D
// (G = Psi^H Psi, S x S) the determinant lemma and the Woodbury identity give
//   log det C = (Nz - S) log eta_bar + log det A,
//   e^H C^-1 e = (|e|^2 - rhs^H A^-1 rhs) / eta_bar,   rhs = D Psi^H e,
// and both come out of one LDL^H elimination of A: log det A = sum_k log piv_k and
// rhs^H A^-1 rhs = sum_k |rhs_k^(k)|^2 / piv_k (forward substitution carried along).
//
// Normalised weights need log-likelihood accuracy only where the weight is not
// negligible: a particle more than Delta nats below the best carries at most e^-Delta
// of the best weight, so an FP32 error of a nat there changes no weight by more than
// e^-Delta relative to the largest.  Each particle's FP32 value therefore comes with
// a bound err_p on its error (pivot cancellation: ~8 eps A_kk / piv_k per pivot; the
// difference |e|^2 - rhs^H A^-1 rhs: a few eps of its terms).  With u_p = log w_p + err_p
// an upper bound of the true log-weight and L the largest lower bound over the particles,
// the FP32 weight of p is off by at most e^(u_p - L) (e^err_p - 1) of the largest weight;
// k_iota_select queues for k_iota_blk (the float-float evaluation) every particle for
// which that bound reaches e^-Delta, so the P particles left in FP32 move the
// normalisation by at most P e^-Delta.
#include "bp_internal.cuh"
#include "bp_kernels.cuh"

namespace bp {

constexpr int IOTA_BULK_T = 64;              // 8 x 8 threads: row residue tr, column residue tc
constexpr int IOTA_BULK_PER_SM = 6;
constexpr float IOTA_ERR_PER_RATIO = 4.0e-6f;   // nats per unit of sum_k A_kk / piv_k (8 eps, x8 margin)
constexpr float IOTA_ERR_PER_ENERGY = 1.0e-6f;  // nats per noise unit of |e|^2 + rhs^H A^-1 rhs (16 eps)
constexpr double IOTA_SELECT_NATS = 24.0;       // Delta: P e^-Delta = 4e-6 at P = 1e5, 1e-5 at 2.6e5

// shared memory (bytes): e [Nz], factors [S][nst], published columns [3][SB], y [SB],
// A pi mu [SB], A pi mu b' [S][Nf | 1], a_y a_z [S][Nm | 1] (float2); d A [SB], diagonal [SB],
// reductions [8] (float)
__host__ __device__ inline size_t iota_bulk_smem(int S, int nst, int Nz, int SB, int Nf, int Nm) {
    return ((size_t)Nz + (size_t)S * nst + 5 * (size_t)SB + (size_t)S * ((Nf | 1) + (Nm | 1))) * sizeof(float2) +
           (2 * (size_t)SB + 8) * sizeof(float);
}

__device__ __forceinline__ void cfma_c(float2& acc, float2 a, float2 b) {   // acc += conj(a) b
    acc.x = fmaf(a.x, b.x, fmaf(a.y, b.y, acc.x));
    acc.y = fmaf(a.x, b.y, fmaf(-a.y, b.x, acc.y));
}
__device__ __forceinline__ void cfms_c(float2& acc, float2 a, float2 b) {   // acc -= a conj(b)
    acc.x = fmaf(-a.x, b.x, fmaf(-a.y, b.y, acc.x));
    acc.y = fmaf(-a.y, b.x, fmaf(a.x, b.y, acc.y));
}

// One block per particle (grid-stride), 64 threads.  The lower triangle of A (S <= 8 NB)
// is held in registers: thread (tr, tc) owns the entries (8 ia + tr, 8 ib + tc), ia >= ib,
// so every thread keeps about S^2 / 128 of them and the trailing work stays balanced as
// the elimination proceeds.  Column k of the elimination is published in shared memory
// by its owners one step ahead (triple-buffered), so each step takes one barrier.
template <int NB>
__global__ void __launch_bounds__(IOTA_BULK_T, IOTA_BULK_PER_SM) k_iota_bulk(DevGeom G, DevParams Pm, DevState D, int S,
                                                                             const float* z) {
    constexpr int SB = 8 * NB;
    constexpr int NSL = NB * (NB + 1) / 2;
    extern __shared__ float4 smq[];
    const int t = threadIdx.x, tr = t & 7, tc = t >> 3;
    const int P = Pm.P, J = G.J, Nz = G.Nz, Nf = G.Nf, My = G.My, Mz = G.Mz, Nm = My * Mz;
    const int nst = (Nf + My + Mz) | 1;   // odd row stride of the factors (bank spread)
    float2* es = reinterpret_cast<float2*>(smq);        // [Nz]   z, then e
    float2* fac = es + Nz;                                // [S][nst] b', a_y, a_z
    float2* pub = fac + (size_t)S * nst;                  // [3][SB] published columns
    float2* yb = pub + 3 * SB;                            // [SB]   y_k = rhs_k^(k) / piv_k
    float2* mt = yb + SB;                                 // [SB]   A_s pi_s mu_s
    const int ust = Nf | 1, cst = Nm | 1;                 // odd row strides (bank spread)
    float2* ub = mt + SB;                                 // [S][ust] A_s pi_s mu_s b'_sf
    float2* cb2 = ub + (size_t)S * ust;                   // [S][cst] a_sy a_sm
    float* dA = reinterpret_cast<float*>(cb2 + (size_t)S * cst);   // [SB]   d_s A_s
    float* dg0 = dA + SB;                                 // [SB]   A_kk before the elimination
    float* red = dg0 + SB;                                // [8]
    const float* phi = D.phi[D.cur];
    // entries of the published columns above the diagonal are read (into entries of
    // A that do not exist) before any owner writes them: start them at zero
    for (int i = t; i < 3 * SB; i += IOTA_BULK_T) pub[i] = make_float2(0.f, 0.f);
    for (int p = blockIdx.x; p < P; p += gridDim.x) {
        double total = 0.0;
        float err = 0.f;
        bool broke = false;
        for (int j = 0; j < J; ++j) {
            __syncthreads();   // the previous (p, j) is done with shared memory
            for (int k = t; k < Nz; k += IOTA_BULK_T) es[k] = make_float2(z[2 * (j * Nz + k)], z[2 * (j * Nz + k) + 1]);
            const double eb = D.eta_bar[j];
            const float ebf = (float)eb;
            if (t < SB) {
                float2 mts = make_float2(0.f, 0.f);
                float das = 0.f;
                if (t < S) {
                    const float* ph = phi + (size_t)t * 6 * P;
                    float2* fs = fac + (size_t)t * nst;
                    const size_t gi = ((size_t)t * J + j) * P + p;
                    const float A = factors_from_geo_folded(G, D.geo[gi], D.geo_lo[gi], fs, fs + Nf, fs + Nf + My, 1);
                    const float pi = (float)(D.zeta[t * J + j] * D.W[t]);
                    const float gm = ph[3 * (size_t)P + p], mr = ph[4 * (size_t)P + p], mi = ph[5 * (size_t)P + p];
                    const float d = sqrtf(fmaxf(pi * (gm + (mr * mr + mi * mi) * (1.0f - pi)), 0.0f));
                    mts = make_float2(A * pi * mr, A * pi * mi);
                    das = d * A;
                }
                mt[t] = mts;
                dA[t] = das;
            }
            __syncthreads();
            // Kronecker parts of the steering vectors: psi'_s[f, (y, m)] = b'_sf (a_sy a_sm)
            for (int i = t; i < S * Nf; i += IOTA_BULK_T) {
                const int s = i / Nf, f = i - s * Nf;
                ub[(size_t)s * ust + f] = cmul(mt[s], fac[(size_t)s * nst + f]);
            }
            for (int i = t; i < S * Nm; i += IOTA_BULK_T) {
                const int s = i / Nm, ym = i - s * Nm, y = ym / Mz, m = ym - y * Mz;
                const float2* fs = fac + (size_t)s * nst;
                cb2[(size_t)s * cst + ym] = cmul(fs[Nf + y], fs[Nf + My + m]);
            }
            __syncthreads();
            // e = z - sum_s (A pi mu b')_sf (a_y a_z)_s,ym, element-wise; |e|^2
            float ee = 0.f;
            for (int k = t; k < Nz; k += IOTA_BULK_T) {
                const int f = k / Nm, ym = k - f * Nm;
                float2 acc = es[k];
                for (int s = 0; s < S; ++s) {
                    const float2 u = ub[(size_t)s * ust + f], c = cb2[(size_t)s * cst + ym];
                    acc.x = fmaf(-u.x, c.x, fmaf(u.y, c.y, acc.x));
                    acc.y = fmaf(-u.x, c.y, fmaf(-u.y, c.x, acc.y));
                }
                es[k] = acc;
                ee = fmaf(acc.x, acc.x, fmaf(acc.y, acc.y, ee));
            }
            ee = warp_sum_f(ee);
            if ((t & 31) == 0) red[t >> 5] = ee;
            __syncthreads();
            // rhs_a = d_a A_a psi'_a^H e (thread a)
            float2 rhs = make_float2(0.f, 0.f);
            if (t < S) {
                const float2* fs = fac + (size_t)t * nst;
                const float2* cs = cb2 + (size_t)t * cst;
                float2 g = make_float2(0.f, 0.f);
                for (int f = 0; f < Nf; ++f) {
                    float2 acc = make_float2(0.f, 0.f);
                    const float2* ef = es + f * Nm;
                    for (int ym = 0; ym < Nm; ++ym) cfma_c(acc, cs[ym], ef[ym]);
                    cfma_c(g, fs[f], acc);
                }
                rhs = make_float2(dA[t] * g.x, dA[t] * g.y);
            }
            // Gram G'_ab = (sum_f conj b'_af b'_bf)(sum_y conj a_ay a_by)(sum_m conj a_am a_bm) of this
            // thread's entries; rows a = 8 ia + tr, columns b = 8 ib + tc, slot ia (ia + 1) / 2 + ib
            float2 A[NSL];
            #pragma unroll
            for (int q = 0; q < NSL; ++q) A[q] = make_float2(0.f, 0.f);
            for (int f = 0; f < Nf; ++f) {
                float2 ra[NB], cb[NB];
                #pragma unroll
                for (int i = 0; i < NB; ++i) {
                    const int a = 8 * i + tr, b = 8 * i + tc;
                    ra[i] = (a < S) ? fac[(size_t)a * nst + f] : make_float2(0.f, 0.f);
                    cb[i] = (b < S) ? fac[(size_t)b * nst + f] : make_float2(0.f, 0.f);
                }
                #pragma unroll
                for (int ia = 0; ia < NB; ++ia) {
                    #pragma unroll
                    for (int ib = 0; ib <= ia; ++ib) cfma_c(A[ia * (ia + 1) / 2 + ib], ra[ia], cb[ib]);
                }
            }
            // the antenna factors, two rows of slots at a time (rows c and NB - 1 - c: NB + 1 slots)
            #pragma unroll
            for (int c = 0; c < (NB + 1) / 2; ++c) {
                const int i0 = c, i1 = NB - 1 - c;
                const bool two = i1 != i0;
                float2 sy[NB + 1], sz[NB + 1];
                #pragma unroll
                for (int q = 0; q <= NB; ++q) sy[q] = sz[q] = make_float2(0.f, 0.f);
                for (int u = 0; u < My + Mz; ++u) {
                    const int off = Nf + u;
                    const int a0 = 8 * i0 + tr, a1 = 8 * i1 + tr;
                    const float2 r0 = (a0 < S) ? fac[(size_t)a0 * nst + off] : make_float2(0.f, 0.f);
                    const float2 r1 = (a1 < S) ? fac[(size_t)a1 * nst + off] : make_float2(0.f, 0.f);
                    float2 cb[NB];
                    #pragma unroll
                    for (int i = 0; i < NB; ++i) {
                        const int b = 8 * i + tc;
                        cb[i] = (b < S) ? fac[(size_t)b * nst + off] : make_float2(0.f, 0.f);
                    }
                    if (u < My) {
                        #pragma unroll
                        for (int ib = 0; ib <= i0; ++ib) cfma_c(sy[ib], r0, cb[ib]);
                        if (two) {
                            #pragma unroll
                            for (int ib = 0; ib <= i1; ++ib) cfma_c(sy[i0 + 1 + ib], r1, cb[ib]);
                        }
                    } else {
                        #pragma unroll
                        for (int ib = 0; ib <= i0; ++ib) cfma_c(sz[ib], r0, cb[ib]);
                        if (two) {
                            #pragma unroll
                            for (int ib = 0; ib <= i1; ++ib) cfma_c(sz[i0 + 1 + ib], r1, cb[ib]);
                        }
                    }
                }
                #pragma unroll
                for (int ib = 0; ib <= i0; ++ib) {
                    float2& v = A[i0 * (i0 + 1) / 2 + ib];
                    v = cmul(v, cmul(sy[ib], sz[ib]));
                }
                if (two) {
                    #pragma unroll
                    for (int ib = 0; ib <= i1; ++ib) {
                        float2& v = A[i1 * (i1 + 1) / 2 + ib];
                        v = cmul(v, cmul(sy[i0 + 1 + ib], sz[i0 + 1 + ib]));
                    }
                }
            }
            // A = eta_bar I + (d A)_a (d A)_b G'_ab; rows and columns beyond S are the identity
            #pragma unroll
            for (int ia = 0; ia < NB; ++ia) {
                #pragma unroll
                for (int ib = 0; ib <= ia; ++ib) {
                    const int a = 8 * ia + tr, b = 8 * ib + tc;
                    float2& v = A[ia * (ia + 1) / 2 + ib];
                    if (a >= S || b >= S) {
                        v = make_float2(a == b ? 1.f : 0.f, 0.f);
                    } else {
                        const float sc = dA[a] * dA[b];
                        v = make_float2(sc * v.x, sc * v.y);
                        if (a == b) v = make_float2(v.x + ebf, 0.f);
                    }
                    if (a == b) dg0[a] = v.x;
                    if (ib == 0 && tc == 0) pub[a] = v;   // column 0 for the first step
                }
            }
            __syncthreads();
            const float ee_all = red[0] + red[1];
            // LDL^H elimination: step k = 8 K + r subtracts A_ak conj(A_bk) / piv_k from the
            // trailing entries (b > k); the forward substitution runs one column behind
            float yy = 0.f;                   // sum over this thread's k of |rhs_k^(k)|^2 / piv_k
            float dm = 1.f, rsum = 0.f, pmin = 3.0e38f;
            int de = 0;
            int k = 0, cur = 0;
            #pragma unroll
            for (int K = 0; K < NB; ++K) {
                for (int r = 0; r < 8; ++r, ++k) {
                    if (k >= S) break;        // uniform over the block
                    const int prv = (cur + 2) % 3, nxt = (cur + 1) % 3;
                    const float2* col = pub + cur * SB;
                    const float piv = col[k].x;
                    const float ipiv = 1.0f / piv;
                    if (k > 0 && t >= k && t < S) {   // column k - 1 into rhs_t
                        const float2 a = pub[prv * SB + t], y = yb[k - 1];
                        rhs.x -= a.x * y.x - a.y * y.y;
                        rhs.y -= a.x * y.y + a.y * y.x;
                    }
                    if (t == k) {
                        yb[k] = make_float2(rhs.x * ipiv, rhs.y * ipiv);
                        yy = fmaf(fmaf(rhs.x, rhs.x, rhs.y * rhs.y), ipiv, yy);
                    }
                    if (t == 0) {
                        int e2;
                        dm = frexpf(dm * piv, &e2);
                        de += e2;
                        rsum += dg0[k] * ipiv;
                        pmin = fminf(pmin, piv);
                    }
                    float2 xa[NB], cc[NB];
                    #pragma unroll
                    for (int i = K; i < NB; ++i) {
                        const float2 va = col[8 * i + tr];
                        xa[i] = make_float2(va.x * ipiv, va.y * ipiv);
                        cc[i] = col[8 * i + tc];
                    }
                    #pragma unroll
                    for (int ia = K; ia < NB; ++ia) {
                        #pragma unroll
                        for (int ib = K; ib <= ia; ++ib) {
                            if (ib > K || tc > r) cfms_c(A[ia * (ia + 1) / 2 + ib], xa[ia], cc[ib]);
                        }
                    }
                    // owners of column k + 1 publish it for the next step
                    float2* ncol = pub + nxt * SB;
                    if (r < 7) {
                        if (tc == r + 1) {
                            #pragma unroll
                            for (int ia = K; ia < NB; ++ia)
                                if (8 * ia + tr > k) ncol[8 * ia + tr] = A[ia * (ia + 1) / 2 + K];
                        }
                    } else if (K + 1 < NB) {
                        if (tc == 0) {
                            #pragma unroll
                            for (int ia = K + 1; ia < NB; ++ia) ncol[8 * ia + tr] = A[ia * (ia + 1) / 2 + (K + 1 < NB ? K + 1 : 0)];
                        }
                    }
                    cur = nxt;
                    __syncthreads();
                }
            }
            yy = warp_sum_f(yy);
            if ((t & 31) == 0) red[2 + (t >> 5)] = yy;
            __syncthreads();
            if (t == 0) {
                const double vv = (double)red[2] + (double)red[3];
                const double q = (double)ee_all - vv;           // eta_bar e^H C^-1 e
                const double logdet = log((double)dm) + (double)de * 0.69314718055994530942;
                const double lg = log(eb);
                total += -q / eb - logdet - (double)(Nz - S) * lg - (double)Nz * 1.14472988584940017414;
                const float eq = IOTA_ERR_PER_ENERGY * (float)(((double)ee_all + vv) / eb);
                err += IOTA_ERR_PER_RATIO * rsum + eq;
                // every pivot of eta_bar I + D G D is at least eta_bar, and q >= 0: anything
                // else is a breakdown of the FP32 elimination
                if (!(pmin > 0.5f * ebf) || !(q / eb > -(double)eq) || !isfinite(total)) broke = true;
            }
        }
        if (t == 0) {
            D.lw_x[p] = total;
            D.iota_err[p] = broke ? INFINITY : err;
        }
    }
}

// ---------------------------------------------------------------- selection
// Doubles as order-preserving unsigned keys for atomicMax (0 is below every key).
__device__ inline unsigned long long dkey(double v) {
    const unsigned long long b = (unsigned long long)__double_as_longlong(v);
    return (b >> 63) ? ~b : (b | 0x8000000000000000ull);
}
__device__ inline double dkey_value(unsigned long long k) {
    if (k == 0ull) return -INFINITY;
    const unsigned long long b = (k >> 63) ? (k & 0x7fffffffffffffffull) : ~k;
    return __longlong_as_double((long long)b);
}

// largest lower bound of log w_beta + log iota~ over the particles
__global__ void __launch_bounds__(256) k_iota_maxlow(DevParams Pm, DevState D) {
    double m = -INFINITY;
    for (int p = blockIdx.x * blockDim.x + threadIdx.x; p < Pm.P; p += gridDim.x * blockDim.x) {
        const double v = log(D.w_x[p]) + D.lw_x[p] - (double)D.iota_err[p];
        if (isfinite(v)) m = fmax(m, v);
    }
    m = warp_max_d(m);
    __shared__ double wm[8];
    if ((threadIdx.x & 31) == 0) wm[threadIdx.x >> 5] = m;
    __syncthreads();
    if (threadIdx.x == 0) {
        for (int w = 1; w < (int)(blockDim.x >> 5); ++w) m = fmax(m, wm[w]);
        if (isfinite(m)) atomicMax(D.iota_key, dkey(m));
    }
}

// queue for the float-float path every particle of non-zero prior weight whose weight
// error bound e^(u_p - L) (e^err_p - 1) reaches e^-Delta of the largest weight, or whose
// value or bound is not finite (a breakdown of the FP32 elimination)
__global__ void __launch_bounds__(256) k_iota_select(DevParams Pm, DevState D) {
    const double lo = dkey_value(*D.iota_key) - IOTA_SELECT_NATS;
    for (int p = blockIdx.x * blockDim.x + threadIdx.x; p < Pm.P; p += gridDim.x * blockDim.x) {
        const double w = D.w_x[p];
        if (!(w > 0.0)) continue;
        const double l = D.lw_x[p];
        const double e = (double)D.iota_err[p];
        const double lx = e > 30.0 ? e : log(expm1(e));   // log(e^err - 1)
        if (!isfinite(l) || !isfinite(e) || log(w) + l + e + lx >= lo) {
            const int slot = atomicAdd(&D.flags[0], 1);
            if (bp_in_range(slot, Pm.P, D.kerr)) D.flags[1 + slot] = p;
        }
    }
}

template <int NB>
static void launch_bulk_nb(const DevGeom& G, const DevParams& Pm, const DevState& D, int S, const float* z,
                           cudaStream_t st) {
    const int nst = (G.Nf + G.My + G.Mz) | 1;
    const size_t smem = iota_bulk_smem(S, nst, G.Nz, 8 * NB, G.Nf, G.My * G.Mz);
    smem_allow_max((const void*)k_iota_bulk<NB>);
    int sms = 0, dev = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    const int blocks = std::min(Pm.P, std::max(1, sms) * IOTA_BULK_PER_SM * 8);
    k_iota_bulk<NB><<<blocks, IOTA_BULK_T, smem, st>>>(G, Pm, D, S, z);
}

// FP32 likelihood of every particle, then the selection for k_iota_blk (3 launches)
int launch_iota_bulk(const DevGeom& G, const DevParams& Pm, const DevState& D, int S, const float* z, cudaStream_t st) {
    cudaMemsetAsync(D.flags, 0, sizeof(int), st);
    cudaMemsetAsync(D.iota_key, 0, sizeof(unsigned long long), st);
    if (S <= 32) launch_bulk_nb<4>(G, Pm, D, S, z, st);
    else launch_bulk_nb<8>(G, Pm, D, S, z, st);
    const int nb = std::min((Pm.P + 255) / 256, 4 * 152);
    k_iota_maxlow<<<nb, 256, 0, st>>>(Pm, D);
    k_iota_select<<<nb, 256, 0, st>>>(Pm, D);
    return 3;
}

size_t iota_bulk_smem_bytes(const DevGeom& G, int S) {
    return iota_bulk_smem(S, (G.Nf + G.My + G.Mz) | 1, G.Nz, S <= 32 ? 32 : 64, G.Nf, G.My * G.Mz);
}

}  // namespace bp
